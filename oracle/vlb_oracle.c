/*
 * vlb_oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY; see vlb_oracle.h).
 *
 * Written from the paper (arXiv 2209.14889) in its notation and order; slow on purpose:
 * every stage is a full-lattice loop in natural (y, x) order, no blocking or fusion.
 * Readings of points the paper leaves open are marked "Reading:" where they are used.
 */
#include "vlb_oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* D2Q9 lattice (Sec. II A: d = 2, N_LB = 9). */
static const int cxs[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int cys[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int opp[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static double wn(int n) { return n == 0 ? 4.0 / 9.0 : (n < 5 ? 1.0 / 9.0 : 1.0 / 36.0); }

static const double PI = 3.14159265358979323846;

/* ------------------------------------------------------------------------------------ */
/* Lattice indexing and boundary rules                                                   */
/* ------------------------------------------------------------------------------------ */

static int wrapi(int i, int n) { i %= n; return i < 0 ? i + n : i; }

/* Minimum-image difference on a periodic axis of length n. */
static double minimg(double d, int n)
{
    double L = (double)n;
    d = fmod(d, L);
    if (d >= 0.5 * L) d -= L;
    if (d < -0.5 * L) d += L;
    return d;
}

enum { BC_NEUMANN = 0, BC_DIRICHLET0 = 1 };

/*
 * Value of component field f at (x, y) with the boundary rule of App. C.
 * Each axis is periodic unless it has walls (walls_x, walls_y), which sit half-way between
 * nodes at -1/2 and n - 1/2; a ghost node beyond a wall mirrors its image: zero-gradient
 * (Neumann) fields copy it, zero-value (Dirichlet) fields negate it (once per mirror).
 * Reading: the paper names the BC types only; mirroring about the half-way wall is the
 * second-order ghost-node form of each.
 */
static double at(const orc_params* p, const double* f, int x, int y, int bc)
{
    int nx = p->nx, ny = p->ny;
    double s = 1.0;
    if (!p->walls_x) x = wrapi(x, nx);
    while (x < 0 || x >= nx) {
        if (x < 0) x = -1 - x; else x = 2 * nx - 1 - x;
        if (bc == BC_DIRICHLET0) s = -s;
    }
    if (!p->walls_y) y = wrapi(y, ny);
    while (y < 0 || y >= ny) {
        if (y < 0) y = -1 - y; else y = 2 * ny - 1 - y;
        if (bc == BC_DIRICHLET0) s = -s;
    }
    return s * f[(size_t)y * nx + x];
}

/* Central first differences and the 5-point Laplacian (second order, Reading Q4). */
static double Dx(const orc_params* p, const double* f, int x, int y, int bc)
{ return 0.5 * (at(p, f, x + 1, y, bc) - at(p, f, x - 1, y, bc)); }
static double Dy(const orc_params* p, const double* f, int x, int y, int bc)
{ return 0.5 * (at(p, f, x, y + 1, bc) - at(p, f, x, y - 1, bc)); }
static double Lap(const orc_params* p, const double* f, int x, int y, int bc)
{
    return at(p, f, x + 1, y, bc) + at(p, f, x - 1, y, bc) + at(p, f, x, y + 1, bc)
         + at(p, f, x, y - 1, bc) - 4.0 * at(p, f, x, y, bc);
}

/* ------------------------------------------------------------------------------------ */
/* Stiffness tensor C~(P)  (Sec. II C 2-3, App. B)                                       */
/* ------------------------------------------------------------------------------------ */

double orc_bessel_i(int n, double k)
{
    /* I_n(k) = sum_m (k/2)^(2m+n) / (m! (m+n)!) */
    double half = 0.5 * k, term = 1.0, sum;
    for (int j = 1; j <= n; ++j) term *= half / j;           /* (k/2)^n / n! */
    sum = term;
    for (int m = 1; m < 1000; ++m) {
        term *= half * half / ((double)m * (double)(m + n));
        sum += term;
        if (term < 1e-18 * sum) break;
    }
    return sum;
}

double orc_k_of_P(double P)
{
    /* Eq. Pk: P(k) = I1(k)/I0(k), increasing from 0 to 1.  Newton on k with a bisection
     * bracket; dP/dk = 1 - P/k - P^2. */
    if (P <= 0.0) return 0.0;
    double lo = 0.0, hi = 1.0;
    while (orc_bessel_i(1, hi) / orc_bessel_i(0, hi) < P) { lo = hi; hi *= 2.0; }
    double k = 2.0 * P / (1.0 - P * P);                      /* small-k estimate */
    if (k <= lo || k >= hi) k = 0.5 * (lo + hi);
    for (int it = 0; it < 200; ++it) {
        double r = orc_bessel_i(1, k) / orc_bessel_i(0, k);
        double g = r - P;
        if (g > 0) hi = k; else lo = k;
        double d = 1.0 - r / k - r * r;
        double kn = k - g / d;
        if (!(kn > lo && kn < hi)) kn = 0.5 * (lo + hi);
        if (fabs(kn - k) <= 1e-15 * (1.0 + k)) { k = kn; break; }
        k = kn;
    }
    return k;
}

void orc_stiffness(const orc_params* p, double Px, double Py, double* C)
{
    /* App. B closed form, with the bracket (k(k^2+24) I0 - 8(k^2+6) I1)/k^3 written as the
     * identical I4(k) (recurrence I_{n+1} = I_{n-1} - (2n/k) I_n), which does not cancel.
     * theta_P = polar angle of P; k from |P| capped at P_cap (Sec. II C 3). */
    double K11 = p->K1111, K12 = p->K1122, K22 = p->K2222, K66 = p->K1212;
    double S = 3 * K11 + 2 * K12 + 4 * K66 + 3 * K22;
    double dK = K11 - K22;
    double X = K11 - 2 * K12 - 4 * K66 + K22;
    double Pm = sqrt(Px * Px + Py * Py);
    double pc = Pm < p->P_cap ? Pm : p->P_cap;
    double r2 = 0.0, r4 = 0.0;
    if (pc > 0.0) {
        double k = orc_k_of_P(pc);
        double I0 = orc_bessel_i(0, k);
        r2 = orc_bessel_i(2, k) / I0;
        r4 = orc_bessel_i(4, k) / I0;
    }
    double th = atan2(Py, Px);
    double c2 = cos(2 * th), s2 = sin(2 * th), c4 = cos(4 * th), s4 = sin(4 * th);
    double C11 = (S + 4 * r2 * dK * c2 + r4 * X * c4) / 8.0;
    double C12 = (K11 + 6 * K12 - 4 * K66 + K22 - r4 * X * c4) / 8.0;
    double C13 = (r4 * X * s4 + 2 * r2 * dK * s2) / 4.0;
    double C22 = C11 - r2 * dK * c2;
    double C23 = (2 * r2 * dK * s2 - r4 * X * s4) / 4.0;
    double C33 = (K11 - 2 * K12 + 4 * K66 + K22 - r4 * X * c4) / 4.0;
    C[0] = C11;       C[1] = C12;       C[2] = C13;
    C[3] = C12;       C[4] = C22;       C[5] = C23;
    C[6] = C13 / 2.0; C[7] = C23 / 2.0; C[8] = C33;
}

/* ------------------------------------------------------------------------------------ */
/* Immersed boundary (App. A)                                                            */
/* ------------------------------------------------------------------------------------ */

double orc_phi(double r)
{
    double a = fabs(r);
    return a < 2.0 ? 0.25 * (1.0 + cos(PI * r / 2.0)) : 0.0;
}

double orc_ring_energy(const orc_ring* g, const double* X)
{
    int N = g->n_nodes;
    double U = 0.0, cx = 0.0, cy = 0.0;
    for (int a = 0; a < N; ++a) {
        int b = (a + 1) % N, z = (a + N - 1) % N;
        double dx = X[2 * b] - X[2 * a], dy = X[2 * b + 1] - X[2 * a + 1];
        double l = sqrt(dx * dx + dy * dy);
        U += 0.5 * g->k_spring * (l - g->l_eq) * (l - g->l_eq);
        double px = X[2 * z] - X[2 * a], py = X[2 * z + 1] - X[2 * a + 1];
        double qx = X[2 * b] - X[2 * a], qy = X[2 * b + 1] - X[2 * a + 1];
        double cg = (px * qx + py * qy) / (sqrt(px * px + py * py) * sqrt(qx * qx + qy * qy));
        /* u_angle = eps (1 - cos(pi - gamma)) = eps (1 + cos gamma) */
        U += g->eps_angle * (1.0 + cg);
        cx += X[2 * a]; cy += X[2 * a + 1];
    }
    /* The constant pull F on R_com (reading Q15), potential -F . R_com, and the harmonic trap
     * of Eq. Utrap, k_trap / 2 |R_ext - R_com|^2 (R_com the plain mean of the positions). */
    U -= g->pull_x * cx / N + g->pull_y * cy / N;
    const double ex = g->trap_x - cx / N, ey = g->trap_y - cy / N;
    U += 0.5 * g->trap_k * (ex * ex + ey * ey);
    return U;
}

void orc_node_forces(const orc_ring* g, const double* X, double* f)
{
    int N = g->n_nodes;
    for (int a = 0; a < 2 * N; ++a) f[a] = 0.0;
    for (int a = 0; a < N; ++a) {
        /* spring on the edge (a, a+1) */
        int b = (a + 1) % N;
        double dx = X[2 * b] - X[2 * a], dy = X[2 * b + 1] - X[2 * a + 1];
        double l = sqrt(dx * dx + dy * dy);
        double T = g->k_spring * (l - g->l_eq);
        f[2 * a] += T * dx / l;     f[2 * a + 1] += T * dy / l;
        f[2 * b] -= T * dx / l;     f[2 * b + 1] -= T * dy / l;
    }
    for (int a = 0; a < N; ++a) {
        /* angle term at node a: u = eps (1 + cos gamma_a), gamma_a between the edges */
        int z = (a + N - 1) % N, b = (a + 1) % N;
        double px = X[2 * z] - X[2 * a], py = X[2 * z + 1] - X[2 * a + 1];
        double qx = X[2 * b] - X[2 * a], qy = X[2 * b + 1] - X[2 * a + 1];
        double lp = sqrt(px * px + py * py), lq = sqrt(qx * qx + qy * qy);
        double c = (px * qx + py * qy) / (lp * lq);
        double dcdpx = qx / (lp * lq) - c * px / (lp * lp);
        double dcdpy = qy / (lp * lq) - c * py / (lp * lp);
        double dcdqx = px / (lp * lq) - c * qx / (lq * lq);
        double dcdqy = py / (lp * lq) - c * qy / (lq * lq);
        double e = g->eps_angle;
        f[2 * z] -= e * dcdpx;  f[2 * z + 1] -= e * dcdpy;
        f[2 * b] -= e * dcdqx;  f[2 * b + 1] -= e * dcdqy;
        f[2 * a] += e * (dcdpx + dcdqx);  f[2 * a + 1] += e * (dcdpy + dcdqy);
    }
    /* the pull and the trap act on R_com; dR_com / dR_a = 1 / N */
    double cx = 0.0, cy = 0.0;
    for (int a = 0; a < N; ++a) { cx += X[2 * a]; cy += X[2 * a + 1]; }
    cx /= N;
    cy /= N;
    const double tx = g->trap_k * (g->trap_x - cx) / N, ty = g->trap_k * (g->trap_y - cy) / N;
    for (int a = 0; a < N; ++a) {
        f[2 * a] += g->pull_x / N;  f[2 * a + 1] += g->pull_y / N;
        f[2 * a] += tx;  f[2 * a + 1] += ty;
    }
}

void orc_spread(const orc_params* p, int n_nodes, const double* X, const double* f, double* fib)
{
    /* f_IB(r) = sum_a f_a K(R_a - r), K = phi(r_x) phi(r_y) / dx^2.  Only the 4x4 cells with
     * |R_a - r| < 2 per axis carry non-zero weight; nodes are added in index order. */
    int nx = p->nx, ny = p->ny;
    size_t N = (size_t)nx * ny;
    memset(fib, 0, 2 * N * sizeof(double));
    for (int a = 0; a < n_nodes; ++a) {
        int x0 = (int)floor(X[2 * a]), y0 = (int)floor(X[2 * a + 1]);
        for (int y = y0 - 1; y <= y0 + 2; ++y) {
            if (p->walls_y && (y < 0 || y >= ny)) continue;
            for (int x = x0 - 1; x <= x0 + 2; ++x) {
                if (p->walls_x && (x < 0 || x >= nx)) continue;
                double w = orc_phi(minimg(X[2 * a] - x, nx)) * orc_phi(minimg(X[2 * a + 1] - y, ny));
                size_t i = (size_t)wrapi(y, ny) * nx + wrapi(x, nx);
                fib[i] += f[2 * a] * w;
                fib[N + i] += f[2 * a + 1] * w;
            }
        }
    }
}

void orc_interp(const orc_params* p, const double* u, int n_nodes, const double* X, double* V)
{
    /* v(R_a) = sum_r dx^2 v(r) K(R_a - r) (App. A). */
    int nx = p->nx, ny = p->ny;
    size_t N = (size_t)nx * ny;
    for (int a = 0; a < n_nodes; ++a) {
        int x0 = (int)floor(X[2 * a]), y0 = (int)floor(X[2 * a + 1]);
        double vx = 0.0, vy = 0.0;
        for (int y = y0 - 1; y <= y0 + 2; ++y) {
            if (p->walls_y && (y < 0 || y >= ny)) continue;
            for (int x = x0 - 1; x <= x0 + 2; ++x) {
                if (p->walls_x && (x < 0 || x >= nx)) continue;
                double w = orc_phi(minimg(X[2 * a] - x, nx)) * orc_phi(minimg(X[2 * a + 1] - y, ny));
                size_t i = (size_t)wrapi(y, ny) * nx + wrapi(x, nx);
                vx += u[i] * w;
                vy += u[N + i] * w;
            }
        }
        V[2 * a] = vx;
        V[2 * a + 1] = vy;
    }
}

/* ------------------------------------------------------------------------------------ */
/* Fields                                                                                */
/* ------------------------------------------------------------------------------------ */

/* Molecular field h = (alpha + beta |P|^2) P - kappa lap P (Eq. Ffunctional and below). */
static void molecular_field(const orc_params* p, const double* P, int x, int y, double* hx, double* hy)
{
    size_t N = (size_t)p->nx * p->ny;
    double px = at(p, P, x, y, BC_NEUMANN), py = at(p, P + N, x, y, BC_NEUMANN);
    double q = px * px + py * py;
    *hx = (p->alpha + p->beta * q) * px - p->kappa * Lap(p, P, x, y, BC_NEUMANN);
    *hy = (p->alpha + p->beta * q) * py - p->kappa * Lap(p, P + N, x, y, BC_NEUMANN);
}

void orc_forces(const orc_params* p, const orc_ring* rings, int n_rings, const double* sigma,
                const double* P, const double* X, const double* fext, double* F, double* fp)
{
    int nx = p->nx, ny = p->ny;
    size_t N = (size_t)nx * ny;
    double* fib = (double*)calloc(2 * N, sizeof(double));
    double* tmp = (double*)malloc(2 * N * sizeof(double));
    double* sE = (double*)malloc(4 * N * sizeof(double));
    double* h2 = (double*)malloc(2 * N * sizeof(double));

    /* Immersed-boundary force of every ring. */
    const double* Xr = X;
    for (int r = 0; r < n_rings; ++r) {
        int n = rings[r].n_nodes;
        double* fa = (double*)malloc(2 * (size_t)n * sizeof(double));
        orc_node_forces(&rings[r], Xr, fa);
        orc_spread(p, n, Xr, fa, tmp);
        for (size_t i = 0; i < 2 * N; ++i) fib[i] += tmp[i];
        free(fa);
        Xr += 2 * n;
    }

    /* Ericksen stress sigma^E_ij = -1/2 (P_i h_j - h_i P_j) + xi/2 (P_i h_j + h_i P_j)
     *                              - kappa d_i P_k d_j P_k
     * Reading Q7: the printed gradient term carries no kappa; kappa is restored so that
     * the stress has the units of the free-energy density. */
    #pragma omp parallel for
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            size_t i = (size_t)y * nx + x;
            double hx, hy;
            molecular_field(p, P, x, y, &hx, &hy);
            h2[i] = hx; h2[N + i] = hy;
            double px = P[i], py = P[N + i];
            double dxPx = Dx(p, P, x, y, BC_NEUMANN), dyPx = Dy(p, P, x, y, BC_NEUMANN);
            double dxPy = Dx(p, P + N, x, y, BC_NEUMANN), dyPy = Dy(p, P + N, x, y, BC_NEUMANN);
            double xi = p->xi, ka = p->kappa;
            sE[i]         = -0.5 * (px * hx - hx * px) + 0.5 * xi * (px * hx + hx * px)
                            - ka * (dxPx * dxPx + dxPy * dxPy);                       /* xx */
            sE[N + i]     = -0.5 * (px * hy - hx * py) + 0.5 * xi * (px * hy + hx * py)
                            - ka * (dxPx * dyPx + dxPy * dyPy);                       /* xy */
            sE[2 * N + i] = -0.5 * (py * hx - hy * px) + 0.5 * xi * (py * hx + hy * px)
                            - ka * (dyPx * dxPx + dyPy * dxPy);                       /* yx */
            sE[3 * N + i] = -0.5 * (py * hy - hy * py) + 0.5 * xi * (py * hy + hy * py)
                            - ka * (dyPx * dyPx + dyPy * dyPy);                       /* yy */
        }

    #pragma omp parallel for
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            size_t i = (size_t)y * nx + x;
            /* f^p_i = d_j sigma^p_ij (Sec. II B); sigma = (xx, yy, xy) */
            double fpx = Dx(p, sigma, x, y, BC_NEUMANN) + Dy(p, sigma + 2 * N, x, y, BC_NEUMANN);
            double fpy = Dx(p, sigma + 2 * N, x, y, BC_NEUMANN) + Dy(p, sigma + N, x, y, BC_NEUMANN);
            /* f^E_i = d_j sigma^E_ij (Sec. II C 1).  Reading (App. C names no condition for
             * sigma^E): beyond a wall the Ericksen stress is the negated image, i.e. it vanishes
             * at the wall, so the divergence telescopes to zero over a closed box as over a
             * periodic one and the polar field hands no momentum to a free-anchoring wall.  (Its
             * zero-gradient image instead let a grid-scale mode at x walls grow without bound
             * once a flow ran along the wall.) */
            double fex = 0.0, fey = 0.0;
            if (p->ericksen) {
                fex = Dx(p, sE, x, y, BC_DIRICHLET0) + Dy(p, sE + N, x, y, BC_DIRICHLET0);
                fey = Dx(p, sE + 2 * N, x, y, BC_DIRICHLET0) + Dy(p, sE + 3 * N, x, y, BC_DIRICHLET0);
            }
            double ex = fext ? fext[i] : 0.0, ey = fext ? fext[N + i] : 0.0;
            F[i] = fib[i] + fpx + fex + ex;
            F[N + i] = fib[N + i] + fpy + fey + ey;
            if (fp) { fp[i] = fpx; fp[N + i] = fpy; }
        }
    free(fib); free(tmp); free(sE); free(h2);
}

void orc_moments(const orc_params* p, const double* h, const double* F, double* rho, double* u)
{
    /* Eq. rhoDef, Eq. vDef with the Guo half-force correction (Reading Q2). */
    size_t N = (size_t)p->nx * p->ny;
    #pragma omp parallel for
    for (size_t i = 0; i < N; ++i) {
        double r = 0.0, jx = 0.0, jy = 0.0;
        for (int n = 0; n < 9; ++n) {
            double hn = h[n * N + i];
            r += hn; jx += cxs[n] * hn; jy += cys[n] * hn;
        }
        rho[i] = r;
        u[i] = (jx + 0.5 * F[i]) / r;
        u[N + i] = (jy + 0.5 * F[N + i]) / r;
    }
}

/* Velocity gradient G_ij = d_i u_j; Psi = sym part, omega = Omega_xy = (d_x u_y - d_y u_x)/2. */
static void velocity_gradient(const orc_params* p, const double* u, double* psi, double* omega)
{
    int nx = p->nx, ny = p->ny;
    size_t N = (size_t)nx * ny;
    #pragma omp parallel for
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            size_t i = (size_t)y * nx + x;
            double dxux = Dx(p, u, x, y, BC_DIRICHLET0), dyux = Dy(p, u, x, y, BC_DIRICHLET0);
            double dxuy = Dx(p, u + N, x, y, BC_DIRICHLET0), dyuy = Dy(p, u + N, x, y, BC_DIRICHLET0);
            psi[i] = dxux;
            psi[N + i] = dyuy;
            psi[2 * N + i] = 0.5 * (dxuy + dyux);
            omega[i] = 0.5 * (dxuy - dyux);
        }
}

void orc_rhs(const orc_params* p, const double* sigma, const double* P, const double* u,
             const double* psi, const double* omega, int with_diffusion, double* dsigma, double* dP)
{
    int nx = p->nx, ny = p->ny;
    size_t N = (size_t)nx * ny;
    #pragma omp parallel for
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            size_t i = (size_t)y * nx + x;
            double ux = u[i], uy = u[N + i];
            double w = omega[i];
            double ps[3] = {psi[i], psi[N + i], psi[2 * N + i]};
            double s[3] = {sigma[i], sigma[N + i], sigma[2 * N + i]};
            double C[9];
            orc_stiffness(p, P[i], P[N + i], C);
            /* Eq. StiffCons with the Jaumann derivative (Sec. II B):
             * d_t s = -(u.grad) s - (Omega s - s Omega) + C psi - C s / eta_p + D_p lap s
             * (Omega s - s Omega) = (2 w s_xy, -2 w s_xy, w (s_yy - s_xx)). */
            double J[3] = {2.0 * w * s[2], -2.0 * w * s[2], w * (s[1] - s[0])};
            for (int c = 0; c < 3; ++c) {
                const double* sc = sigma + c * N;
                double adv = ux * Dx(p, sc, x, y, BC_NEUMANN) + uy * Dy(p, sc, x, y, BC_NEUMANN);
                double Cpsi = C[3 * c] * ps[0] + C[3 * c + 1] * ps[1] + C[3 * c + 2] * ps[2];
                double Cs = C[3 * c] * s[0] + C[3 * c + 1] * s[1] + C[3 * c + 2] * s[2];
                double dif = with_diffusion ? p->Dp * Lap(p, sc, x, y, BC_NEUMANN) : 0.0;
                dsigma[c * N + i] = -adv - J[c] + Cpsi - Cs / p->eta_p + dif;
            }
            /* Eq. BE: d_t P_i = -(u.grad) P_i - Omega_ik P_k + xi Psi_ik P_k - Gamma h_i */
            double px = P[i], py = P[N + i];
            double hx, hy;
            molecular_field(p, P, x, y, &hx, &hy);
            double advx = ux * Dx(p, P, x, y, BC_NEUMANN) + uy * Dy(p, P, x, y, BC_NEUMANN);
            double advy = ux * Dx(p, P + N, x, y, BC_NEUMANN) + uy * Dy(p, P + N, x, y, BC_NEUMANN);
            dP[i] = -advx - w * py + p->xi * (ps[0] * px + ps[2] * py) - p->Gamma * hx;
            dP[N + i] = -advy + w * px + p->xi * (ps[2] * px + ps[1] * py) - p->Gamma * hy;
        }
}

/* ------------------------------------------------------------------------------------ */
/* One time step                                                                          */
/* ------------------------------------------------------------------------------------ */

int orc_step(const orc_params* p, const orc_ring* rings, int n_rings,
             double* h, double* sigma, double* P, double* X, const double* fext,
             orc_diag* diag, double* frest, double* com)
{
    int nx = p->nx, ny = p->ny;
    size_t N = (size_t)nx * ny;
    int n_total = 0;
    for (int r = 0; r < n_rings; ++r) n_total += rings[r].n_nodes;

    double* F = (double*)malloc(2 * N * sizeof(double));
    double* fp = (double*)malloc(2 * N * sizeof(double));
    double* rho = (double*)malloc(N * sizeof(double));
    double* u = (double*)malloc(2 * N * sizeof(double));
    double* hs = (double*)malloc(9 * N * sizeof(double));
    double* psi = (double*)malloc(3 * N * sizeof(double));
    double* om = (double*)malloc(N * sizeof(double));
    double* ds0 = (double*)malloc(3 * N * sizeof(double));
    double* dP0 = (double*)malloc(2 * N * sizeof(double));
    double* ds1 = (double*)malloc(3 * N * sizeof(double));
    double* dP1 = (double*)malloc(2 * N * sizeof(double));
    double* s1 = (double*)malloc(3 * N * sizeof(double));
    double* P1 = (double*)malloc(2 * N * sizeof(double));
    double* V0 = (double*)malloc(2 * (size_t)(n_total + 1) * sizeof(double));
    double* V1 = (double*)malloc(2 * (size_t)(n_total + 1) * sizeof(double));
    double* Xs = (double*)malloc(2 * (size_t)(n_total + 1) * sizeof(double));
    if (!F || !fp || !rho || !u || !hs || !psi || !om || !ds0 || !dP0 || !ds1 || !dP1 || !s1 ||
        !P1 || !V0 || !V1 || !Xs) return -1;

    /* 1-4. forces of the state at t: f_a, spread, f^p, f^E, F (Fig. 2). */
    orc_forces(p, rings, n_rings, sigma, P, X, fext, F, fp);

    /* 5. moments rho, u (Eq. rhoDef, vDef, Guo half force). */
    orc_moments(p, h, F, rho, u);

    /* diagnostics of the state at t */
    if (diag) {
        double m = 0.0, jx = 0.0, jy = 0.0, fx = 0.0, fy = 0.0;
        for (size_t i = 0; i < N; ++i) {
            m += rho[i] - p->rho0;
            for (int n = 0; n < 9; ++n) { jx += cxs[n] * h[n * N + i]; jy += cys[n] * h[n * N + i]; }
            fx += F[i]; fy += F[N + i];
        }
        diag->mass_excess = m; diag->mom[0] = jx; diag->mom[1] = jy;
        diag->force[0] = fx; diag->force[1] = fy;
    }
    if (frest || com) {
        const double* Xr = X;
        for (int r = 0; r < n_rings; ++r) {
            int n = rings[r].n_nodes;
            if (frest) {
                /* Reading Q17: restoring force = f^p = div sigma^p interpolated to the nodes
                 * with the IB kernel and summed over the ring. */
                orc_interp(p, fp, n, Xr, V0);
                double sx = 0.0, sy = 0.0;
                for (int a = 0; a < n; ++a) { sx += V0[2 * a]; sy += V0[2 * a + 1]; }
                frest[2 * r] = sx; frest[2 * r + 1] = sy;
            }
            if (com) {
                double sx = 0.0, sy = 0.0;
                for (int a = 0; a < n; ++a) { sx += Xr[2 * a]; sy += Xr[2 * a + 1]; }
                sx /= n; sy /= n;
                sx = fmod(sx, (double)nx); if (sx < 0) sx += nx;
                sy = fmod(sy, (double)ny); if (sy < 0) sy += ny;
                com[2 * r] = sx; com[2 * r + 1] = sy;
            }
            Xr += 2 * n;
        }
    }

    /* 6. BGK collision with Guo forcing (Eq. LB, Eq. BGK; Readings Q1, Q2):
     * h* = h - (h - h^eq)/tau + (1 - 1/(2 tau)) w_n [3(c_n - u) + 9 (c_n.u) c_n] . F */
    double tau = p->tau;
    #pragma omp parallel for
    for (size_t i = 0; i < N; ++i) {
        double ux = u[i], uy = u[N + i], r = rho[i], Fx = F[i], Fy = F[N + i];
        double uu = ux * ux + uy * uy;
        for (int n = 0; n < 9; ++n) {
            double cu = cxs[n] * ux + cys[n] * uy;
            double heq = wn(n) * r * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
            double S = (1.0 - 0.5 / tau) * wn(n) *
                       ((3.0 * (cxs[n] - ux) + 9.0 * cu * cxs[n]) * Fx +
                        (3.0 * (cys[n] - uy) + 9.0 * cu * cys[n]) * Fy);
            hs[n * N + i] = h[n * N + i] - (h[n * N + i] - heq) / tau + S;
        }
    }
    /* 7. streaming h_n(r + c_n, t+1) = h*_n(r); half-way bounce-back at walls (App. C): a
     * population whose link crosses a wall returns to its cell as the opposite one. */
    #pragma omp parallel for
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            size_t i = (size_t)y * nx + x;
            for (int n = 0; n < 9; ++n) {
                int xr = x + cxs[n], xd = wrapi(xr, nx), yd = y + cys[n];
                if ((p->walls_y && (yd < 0 || yd >= ny)) || (p->walls_x && (xr < 0 || xr >= nx))) {
                    h[opp[n] * N + i] = hs[n * N + i];
                } else {
                    h[n * N + (size_t)wrapi(yd, ny) * nx + xd] = hs[n * N + i];
                }
            }
        }

    /* 8. velocity gradient of u(t), frozen for the finite-difference updates. */
    velocity_gradient(p, u, psi, om);

    /* 9. predictor-corrector (Reading Q3: Heun) on (sigma, P) jointly. */
    int sub = p->diffusion_substeps;
    orc_rhs(p, sigma, P, u, psi, om, sub == 0, ds0, dP0);
    #pragma omp parallel for
    for (size_t i = 0; i < 3 * N; ++i) s1[i] = sigma[i] + ds0[i];
    #pragma omp parallel for
    for (size_t i = 0; i < 2 * N; ++i) P1[i] = P[i] + dP0[i];
    orc_rhs(p, s1, P1, u, psi, om, sub == 0, ds1, dP1);
    #pragma omp parallel for
    for (size_t i = 0; i < 3 * N; ++i) sigma[i] += 0.5 * (ds0[i] + ds1[i]);
    #pragma omp parallel for
    for (size_t i = 0; i < 2 * N; ++i) P[i] += 0.5 * (dP0[i] + dP1[i]);
    if (sub > 0) {
        /* Reading Q13: explicit stress diffusion beyond the Heun bound, in s sub-steps. */
        orc_params q = *p;
        q.Dp = p->Dp / sub;
        for (int k = 0; k < sub; ++k) {
            #pragma omp parallel for collapse(2)
            for (int c = 0; c < 3; ++c)
                for (int y = 0; y < ny; ++y)
                    for (int x = 0; x < nx; ++x)
                        ds0[c * N + (size_t)y * nx + x] = q.Dp * Lap(&q, sigma + c * N, x, y, BC_NEUMANN);
            #pragma omp parallel for
            for (size_t i = 0; i < 3 * N; ++i) s1[i] = sigma[i] + ds0[i];
            #pragma omp parallel for collapse(2)
            for (int c = 0; c < 3; ++c)
                for (int y = 0; y < ny; ++y)
                    for (int x = 0; x < nx; ++x)
                        ds1[c * N + (size_t)y * nx + x] = q.Dp * Lap(&q, s1 + c * N, x, y, BC_NEUMANN);
            #pragma omp parallel for
            for (size_t i = 0; i < 3 * N; ++i) sigma[i] += 0.5 * (ds0[i] + ds1[i]);
        }
    }

    /* 10. nodes: overdamped advection dR/dt = v(R) by Heun on the frozen u(t) (App. A). */
    if (n_total > 0) {
        orc_interp(p, u, n_total, X, V0);
        for (int a = 0; a < 2 * n_total; ++a) Xs[a] = X[a] + V0[a];
        orc_interp(p, u, n_total, Xs, V1);
        for (int a = 0; a < 2 * n_total; ++a) X[a] += 0.5 * (V0[a] + V1[a]);
    }

    free(F); free(fp); free(rho); free(u); free(hs); free(psi); free(om);
    free(ds0); free(dP0); free(ds1); free(dP1); free(s1); free(P1); free(V0); free(V1); free(Xs);
    return 0;
}
