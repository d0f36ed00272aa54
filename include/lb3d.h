/*
 * lb3d.h -- C ABI of the three-dimensional form of the viscoelastic lattice-Boltzmann step
 * (Floyd, Vaikuntanathan, Dinner, arXiv 2209.14889; the first extension of Sec. IV: the method
 * of Sec. II on a D3Q19 lattice, with the orientation integral of Eq. CTens taken over the unit
 * sphere).
 *
 * What one step computes (Fig. 2, in three dimensions), every stage in CUDA kernels:
 *   1. molecular field h = (alpha + beta |P|^2) P - kappa lap P (Eq. Ffunctional) and the
 *      Ericksen stress sigma^E (Sec. II C 1) of the state at t;
 *   2. F = div sigma^p + div sigma^E + f_ext; moments rho, u with the Guo half force
 *      (Eq. rhoDef, Eq. vDef); BGK collision with the Guo source and streaming (Eq. LB, Eq. BGK);
 *   3. Heun predictor-corrector of sigma^p (Eq. StiffCons, Jaumann derivative) and P (Eq. BE) on
 *      the frozen u(t), with the stiffness C(P) = int g(n) K(n) dOmega over the unit sphere:
 *      g the Fisher density (the maximum-entropy density on the sphere with mean projection |P|,
 *      the three-dimensional counterpart of the von Mises density of Sec. II C 3) and K(n) the
 *      rotation of K^x (Eq. rotate), taken transversely isotropic about the polymer axis.
 * The orientation moments <(n.P^)^2>, <(n.P^)^4> that fix C, combined with K^x into the five
 * coefficients of C:X, are tabulated against |P| on the host in FP64 (8192 intervals up to P_cap);
 * the kernels interpolate them linearly and apply C in its transversely isotropic form about P^.
 *
 * Scope: a periodic box (no immersed boundary: the paper specifies no three-dimensional
 * membrane), FP32 state and arithmetic, FP64 readout sums.  Lattice units dx = dt = 1.
 *
 * Layout in device memory: 28 planes of nx*ny*nz FP32 values, x fastest then y then z:
 * 19 shifted populations d_n = h_n - w_n rho0 (D3Q19: rest, the six faces +x -x +y -y +z -z, the
 * twelve edges (+x+y) (-x-y) (+x-y) (-x+y) (+x+z) (-x-z) (+x-z) (-x+z) (+y+z) (-y-z) (+y-z)
 * (-y+z)), then sigma^p (xx, yy, zz, yz, xz, xy), then dP = P - P_ref (x, y, z).  Two such buffers
 * alternate.
 *
 * Errors: every call returns LB_OK (0) or a negative code of lb.h; lb3d_last_error gives the
 * message.  Handles are not thread-safe; the handle owns all device memory it allocates.
 */
#ifndef LB3D_H
#define LB3D_H
#include <stddef.h>
#include <stdint.h>

#include "lb.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lb3d_params {
    int32_t nx, ny, nz;        /* lattice (each >= 3; nx * ny * nz < 2^31)                    */
    int32_t readout_every;     /* readout period in steps (>= 1)                              */
    double tau, rho0;          /* BGK relaxation time (> 1/2), rest density                   */
    double K1111, K1122, K2222, K1212, K2233;   /* K^x: transversely isotropic about x        */
    double eta_p, Dp;          /* polymer viscosity (> 0), stress diffusion (Eq. StiffCons)   */
    double alpha, beta, xi, Gamma, kappa;      /* Beris-Edwards (Eq. BE, Eq. Ffunctional)     */
    double P_cap;              /* cap on |P| when the concentration is formed (0 < P_cap < 1)  */
    double fext[3];            /* uniform external body force                                 */
    double P_ref[3];           /* uniform reference polarization: P is stored as dP = P - P_ref
                                  (FP32 keeps the deviations; alpha + beta |P|^2 is formed as
                                  (alpha + beta |P_ref|^2) + beta (2 P_ref.dP + |dP|^2), without
                                  the cancellation near |P|^2 = -alpha/beta); 0 is allowed       */
    int32_t ericksen;          /* 1: include f^E in the force                                 */
    int32_t max_samples;       /* rows of the readout ring buffer (>= 1)                      */
} lb3d_params;

typedef struct lb3d_handle lb3d_handle;

/* Field indices of lb3d_readout: 0 rho - rho0, 1-3 u (with the half-force correction), 4-9
 * sigma^p (xx, yy, zz, yz, xz, xy), 10-12 P (= P_ref + dP), 13-31 the shifted populations
 * d_0 .. d_18. */
#define LB3D_FIELD_DRHO 0
#define LB3D_FIELD_U 1
#define LB3D_FIELD_SIGMA 4
#define LB3D_FIELD_P 10
#define LB3D_FIELD_POP0 13
#define LB3D_N_FIELDS 32

/* Allocate a handle on the current CUDA device: LB_EINVAL for bad parameters, LB_EUNSTABLE beyond
 * the explicit Heun bounds (12 D_p <= 2, 12 Gamma kappa <= 2, Gamma |alpha| <= 1), LB_ENOMEM,
 * LB_ECUDA (no device). */
int lb3d_create(const lb3d_params* p, lb3d_handle** out);
void lb3d_destroy(lb3d_handle* h);
const char* lb3d_last_error(const lb3d_handle* h);

/* Initial state: fluid at rest at rho0, sigma^p = 0, P = P_init (host FP64 [3][nz][ny][nx],
 * copied; NULL: P = 0).  Resets the step counter and the readout series. */
int lb3d_init_fields(lb3d_handle* h, const double* P_init);

/* Advance n >= 0 steps (asynchronous on the handle's stream; LB_ESTATE before lb3d_init_fields). */
int lb3d_step(lb3d_handle* h, int64_t n);
/* Wait for the stream; LB_ENONFINITE if a readout sum became NaN/Inf (the flag is cleared). */
int lb3d_sync(lb3d_handle* h);
int64_t lb3d_time(const lb3d_handle* h);

/* Copy one field (FP32, [nz][ny][nx]) of the current state into dst (count >= nx*ny*nz values;
 * dst_is_device: dst is device memory).  Fields 0-3 run a moments pass on the current state. */
int lb3d_readout(lb3d_handle* h, int32_t field, float* dst, size_t count, int32_t dst_is_device);

/* Readout rows of the steps t with t % readout_every == 0 (the most recent max_samples of them,
 * oldest first): (t, mass excess sum (rho - rho0), bare momentum x y z, total force x y z), FP64
 * sums in a fixed order.  dst: host [max_rows][8]; *rows_written gets the count. */
int lb3d_series(lb3d_handle* h, double* dst, int32_t max_rows, int32_t* rows_written);

/* Per-kernel timing: enable = 1 brackets every step with CUDA events; lb3d_kernel_time returns
 * the summed device time (ms) of the steps since timing was enabled and their number. */
int lb3d_timing(lb3d_handle* h, int32_t enable);
int lb3d_kernel_time(lb3d_handle* h, double* ms, int64_t* steps);
/* Kernels launched per step: 4 (Ericksen stress, collision, predictor, corrector), 3 without the
 * Ericksen force. */
int32_t lb3d_launches_per_step(const lb3d_handle* h);

/* The orientation moments behind the kernels' table: (<mu^2>, <mu^4>) of the Fisher density at
 * |P| = P_cap i / 8192, i = 0 .. 8192, as FP32 pairs (dst: 2 * 8193 floats, or NULL to get the
 * entry count).  Returns the number of entries or LB_EINVAL. */
int32_t lb3d_moment_table(double P_cap, float* dst, int32_t max_entries);

/* Algorithmic bytes per cell and step (the state read once and written once: 2 x 28 x 4). */
double lb3d_bytes_per_cell(const lb3d_handle* h);

#ifdef __cplusplus
}
#endif
#endif
