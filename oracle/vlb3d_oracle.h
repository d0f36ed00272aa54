/*
 * vlb3d_oracle.h -- plain FP64 CPU oracle for the three-dimensional form of the viscoelastic
 * lattice-Boltzmann step (Floyd, Vaikuntanathan, Dinner, arXiv 2209.14889): the first
 * extension of Sec. IV, with the D3Q19 lattice and the orientation integral of Eq. CTens taken
 * over the unit sphere numerically.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite and the CPU legs of the benchmark may load
 * this library.  The product path (the CUDA library and its Python binding) never calls it and
 * shares no code with it.
 *
 * Scope: a periodic box with the lattice fields of Sec. II (no immersed boundary: the paper
 * specifies no three-dimensional membrane), and an optional uniform external force.  Units are
 * lattice units: dx = dt = 1, c_s^2 = 1/3.  Fields are stored as [component][z][y][x] with x
 * fastest, FP64; populations are the plain h_n (not shifted).  Symmetric tensors (sigma^p) are
 * stored as the six components (xx, yy, zz, yz, xz, xy).
 *
 * Parity status per function (pins live in tests/test_oracle3d_pins.py):
 *   o3_lattice            pinned (isotropy of the D3Q19 moments up to fourth order)
 *   o3_langevin, o3_k_of_P  pinned (series and closed form; round trip)
 *   o3_orientation_moments  pinned (closed-form recursion of the moments of the Fisher density)
 *   o3_stiffness          pinned (brute-force sphere quadrature of the rotated K^x of Eq. rotate;
 *                         isotropic average; affine case; rotation covariance)
 *   o3_forces             pinned (divergence of sigma^p and sigma^E of a single Fourier mode
 *                         against the analytic derivative, second-order convergence)
 *   o3_step               pinned piecewise (shear-wave decay at nu = (tau - 1/2)/3, exact momentum
 *                         input of a body force, Maxwell shear wave against its linear two-mode
 *                         solution, relaxation of P to |P|^2 = -alpha/beta, conservation); the
 *                         coupled nonlinear run has no closed form: parity unpinned beyond those.
 */
#ifndef VLB3D_ORACLE_H
#define VLB3D_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef struct o3_params {
    int32_t nx, ny, nz;
    int32_t n_quad;                         /* Gauss-Legendre points per panel of the polar integral */
    double tau, rho0;                       /* BGK relaxation time, rest density              */
    double K1111, K1122, K2222, K1212;      /* K^x (Eq. Kmatrix) for polymers along x, extended to */
    double K2233;                           /* three dimensions by transverse isotropy about x */
    double eta_p, Dp;                       /* polymer viscosity, stress diffusion (Eq. StiffCons) */
    double alpha, beta, xi, Gamma, kappa;   /* Beris-Edwards (Eq. BE, Eq. Ffunctional)        */
    double P_cap;                           /* cap on |P| when solving for the concentration k */
    int32_t ericksen, pad_;                 /* 1: include f^E = div sigma^E in the force      */
} o3_params;

/* Diagnostics of the state at time t (the input of the step). */
typedef struct o3_diag {
    double mass_excess;      /* sum_x (rho - rho0)                  */
    double mom[3];           /* sum_x sum_n c_n h_n (bare momentum) */
    double force[3];         /* sum_x F (total body force)          */
} o3_diag;

/* D3Q19 velocities c[19][3] and weights w[19]. */
void o3_lattice(int32_t* c, double* w);

/* Langevin function coth(k) - 1/k: the mean of n.P^ under the Fisher density on the sphere. */
double o3_langevin(double k);
/* Its inverse: the concentration k >= 0 whose Fisher density has mean projection P in [0, 1). */
double o3_k_of_P(double P);
/* n-point Gauss-Legendre nodes x[n] and weights w[n] on [-1, 1]. */
void o3_gauss_legendre(int32_t n, double* x, double* w);
/* <mu^j>, j = 0..4, of mu = n.P^ under the Fisher density exp(k mu) on the unit sphere, by
 * numerical quadrature (the azimuth integrates to 2 pi). */
void o3_orientation_moments(double k, int32_t n_quad, double* m);
/* Stiffness tensor C_ijkl(P), 81 entries (i fastest last: C[((i*3+j)*3+k)*3+l]). */
void o3_stiffness(const o3_params* p, const double* P, double* C);

/* Molecular field h [3][N] and total force F [3][N] of the state (sigma [6][N], P [3][N]);
 * fext: optional uniform force (3 values) or NULL; fp: optional f^p = div sigma^p [3][N]. */
void o3_forces(const o3_params* p, const double* sigma, const double* P, const double* fext,
               double* F, double* h, double* fp);
/* Right-hand sides of Eq. StiffCons and Eq. BE at (sigma, P) with the flow u frozen. */
void o3_rhs(const o3_params* p, const double* sigma, const double* P, const double* u,
            double* dsigma, double* dP);
/* Moments: rho [N] and u [3][N] (Guo half-force). */
void o3_moments(const o3_params* p, const double* h, const double* F, double* rho, double* u);
/* One time step in the order of Fig. 2 (forces, moments, collision and streaming, Heun
 * predictor-corrector of sigma and P on the frozen u); diag (optional) gets the diagnostics of
 * the state at t.  Returns 0, or -1 if memory ran out. */
int o3_step(const o3_params* p, double* h, double* sigma, double* P, const double* fext, o3_diag* diag);

#ifdef __cplusplus
}
#endif
#endif
