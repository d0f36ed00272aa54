/*
 * vlb_oracle.h -- plain FP64 CPU oracle for one time step of the immersed-boundary /
 * lattice-Boltzmann solver of a tensorial viscoelastic fluid (Floyd, Vaikuntanathan,
 * Dinner, arXiv 2209.14889).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load this library.  The product path (the CUDA library and
 * its Python binding) never calls it and shares no code with it.
 *
 * Units are lattice units: dx = dt = 1, c_s^2 = 1/3.  Every field is stored as
 * [component][y][x] with x fastest, FP64.  Populations are the plain h_n (not shifted).
 *
 * Parity status per function (pins live in tests/test_oracle_pins.py):
 *   orc_bessel_i          pinned (library routine, integral representation)
 *   orc_k_of_P            pinned (inverse of Eq. Pk, round trip)
 *   orc_stiffness         pinned (quadrature of Eq. Cdef1 with Eq. qmatrix; 4-index rotation Eq. rotate;
 *                         isotropic limit of Sec. II C; period pi)
 *   orc_phi / spread / interp  pinned (partition of unity, adjointness, force equality)
 *   orc_node_forces       pinned (finite differences of Eq. Const)
 *   orc_step              pinned piecewise (Taylor-Green, Kolmogorov, Poiseuille, stress decay,
 *                         stress diffusion, P relaxation, objectivity, conservation, mirror symmetry,
 *                         the restoring-force readout of a uniform and of a linear polymer force,
 *                         the Heun node advance in a rigid rotation);
 *                         the whole coupled run has no closed form: parity unpinned beyond
 *                         those invariants.
 */
#ifndef VLB_ORACLE_H
#define VLB_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_params {
    int32_t nx, ny;
    double tau, rho0;                       /* BGK relaxation time (Eq. BGK), rest density   */
    double K1111, K1122, K2222, K1212;      /* K^x of Eq. Kmatrix (prefactor absorbed, App. B) */
    double eta_p, Dp;                       /* polymer viscosity, stress diffusion (Eq. StiffCons) */
    double alpha, beta, xi, Gamma, kappa;   /* Beris-Edwards (Eq. BE, Eq. Ffunctional)        */
    double P_cap;                           /* cap on |P| when solving Eq. Pk for k (0.99)   */
    int32_t ericksen;                       /* 1: include f^E = div sigma^E in the force      */
    int32_t walls_y;                        /* 1: halfway bounce-back walls at y=-1/2, ny-1/2 */
    int32_t diffusion_substeps;             /* 0: D_p inside the Heun RHS; s>0: Heun without
                                               diffusion, then s Heun sub-steps of D_p/s      */
    int32_t walls_x;                        /* 1: halfway bounce-back walls at x=-1/2, nx-1/2 */
} orc_params;

typedef struct orc_ring {
    int32_t n_nodes, pad_;
    double k_spring, eps_angle, l_eq;       /* Eq. Const: spring and angle terms              */
    double pull_x, pull_y;                  /* constant total pull force on the ring          */
    double trap_k, trap_x, trap_y;          /* Eq. Utrap at this step: k_trap(t), R_ext(t)    */
} orc_ring;

/* Diagnostics of the state at time t (the input of the step). */
typedef struct orc_diag {
    double mass_excess;      /* sum_x (rho - rho0)                        */
    double mom[2];           /* sum_x sum_n c_n h_n (bare momentum)        */
    double force[2];         /* sum_x F (total body force)                 */
} orc_diag;

/* Modified Bessel function of the first kind I_n(k), n >= 0, by its power series. */
double orc_bessel_i(int n, double k);
/* Solve I1(k)/I0(k) = P for k >= 0 (Eq. Pk), 0 <= P < 1. */
double orc_k_of_P(double P);
/* Stiffness tensor C~(P) in the plain-component basis s = (s11, s22, s12): C[3*r + c]. */
void orc_stiffness(const orc_params* p, double Px, double Py, double* C);
/* Cosine immersed-boundary kernel phi(r) (App. A). */
double orc_phi(double r);
/* Lagrangian node forces f_a = -grad U (Eq. Const without the trap; constant pull). */
void orc_node_forces(const orc_ring* ring, const double* X, double* f);
/* Energy U of one ring (spring + angle + trap + pull potential -F.R_com), for finite-difference pins. */
double orc_ring_energy(const orc_ring* ring, const double* X);
/* Spread node forces onto the lattice: fib[2][ny][nx] is overwritten. */
void orc_spread(const orc_params* p, int n_nodes, const double* X, const double* f, double* fib);
/* Interpolate a 2-component lattice field at node positions: V[2*n]. */
void orc_interp(const orc_params* p, const double* u, int n_nodes, const double* X, double* V);

/* Velocity field u = (sum c h + F/2)/rho and rho, given h and the force field F. */
void orc_moments(const orc_params* p, const double* h, const double* F, double* rho, double* u);
/* Total force density F = f_IB + f^p + f^E (+ fext) of the state. */
void orc_forces(const orc_params* p, const orc_ring* rings, int n_rings, const double* sigma,
                const double* P, const double* X, const double* fext, double* F, double* fp);
/* Right-hand sides of Eq. StiffCons and Eq. BE for frozen u, Psi, omega. */
void orc_rhs(const orc_params* p, const double* sigma, const double* P, const double* u,
             const double* psi, const double* omega, int with_diffusion, double* dsigma, double* dP);

/*
 * One time step t -> t+1 (Fig. 2: every update reads the state at t).
 *   h[9][ny][nx], sigma[3][ny][nx] (xx, yy, xy), P[2][ny][nx], X[2*total_nodes] (unwrapped,
 *   ring after ring), fext[2][ny][nx] or NULL (extra body force, pins only).
 * Optional outputs of the state at t: diag (global sums), frest[2*n_rings] (restoring force
 * sum_a sum_x f^p phi phi), com[2*n_rings] (centre of mass, wrapped into the box).
 * Returns 0, or -1 on allocation failure.
 */
int orc_step(const orc_params* p, const orc_ring* rings, int n_rings,
             double* h, double* sigma, double* P, double* X, const double* fext,
             orc_diag* diag, double* frest, double* com);

#ifdef __cplusplus
}
#endif
#endif
