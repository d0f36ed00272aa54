// lb_internal.h -- device-side data layout and kernel launchers shared by the CUDA sources of
// the solver (not part of the public C ABI; see include/lb.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace vlb {

// Plane order of the stored state: 9 shifted populations d_n = h_n - w_n rho0, then
// sigma^p (xx, yy, xy), then the shifted polarisation dP = P - P_ref (x, y), where P_ref is the
// uniform initial director field P_eq (cos theta_d, sin theta_d) rounded to FP32.  Each plane is
// nx*ny FP32, x fastest.  Storing deviations keeps FP32 resolution where the physics needs it:
// the molecular field depends on alpha + beta |P|^2, which nearly cancels at |P| ~ P_eq.
enum { PL_POP = 0, PL_SXX = 9, PL_SYY = 10, PL_SXY = 11, PL_PX = 12, PL_PY = 13, N_PLANES = 14 };

// C~(P) table: a2(q) = r2/q and a4(q) = r4/q^2 with q = |P|^2, r_n = I_n(k)/I_0(k), k = k(|P|)
// (Eq. Pk), sampled at LUT_N + 1 uniform points of q in [0, q_cap], q_cap = P_cap^2;
// interpolated linearly (relative error <= 3.2e-7 for a4, 2e-8 for a2; read through L1).
// Beyond q_cap: a2 = a2(q_cap) q_cap/q, a4 = a4(q_cap) (q_cap/q)^2 (k is fixed at the cap,
// theta_P still follows P).
constexpr int LUT_N = 4096;

// Per-ring device record.
struct RingDev {
    int n_nodes, node_off;        // nodes [node_off, node_off + n_nodes)
    double k_spring, eps_angle, l_eq, pull_x, pull_y;   // pull per node = pull / n_nodes
    int4 box[2];                  // work box (x0, y0, w, h; wrapped origin) of the steps with even
                                  // and odd t: step t reads box[t & 1], its node update writes the
                                  // other one, so a lattice kernel that advances the nodes while
                                  // its later tiles still run keeps them on the box of step t
    int cap_w, cap_h;             // capacity of the box buffers
    long long box_off;            // offset (floats) of this ring's boxes in the box buffers
    // harmonic trap (Eq. Utrap; trap_k = 0: none): protocol parameters, the initial centre of
    // mass, and the force on each node for the steps with even and odd t (written by the node
    // update of the step before, read by the spreading: the slots alternate like the boxes)
    double trap_k, trap_dx, trap_dy, trap_t_eq, trap_pull, trap_w, trap_x0, trap_y0;
    float2 trap_f[2];
};

__host__ __device__ inline int4 ring_box(const RingDev& R, long long t) { return R.box[t & 1]; }

// Physical constants of the lattice kernel, FP32.
struct Phys {
    float omega;        // 1 / tau
    float guo;          // 1 - 1/(2 tau)
    float rho0;
    float alpha, beta, xi, Gamma, kappa, Dp, inv_eta;
    float prx, pry;     // P_ref (FP32)
    float A0;           // alpha + beta |P_ref|^2, formed in FP64 from the FP32 P_ref
    float kS8;          // (3K1111 + 2K1122 + 4K1212 + 3K2222) / 8
    float kC12;         // (K1111 + 6K1122 - 4K1212 + K2222) / 8
    float kC33;         // (K1111 - 2K1122 + 4K1212 + K2222) / 4
    float dK;           // K1111 - K2222
    float kX;           // K1111 - 2K1122 - 4K1212 + K2222
    float q_cap;
    float lut_scale;    // LUT_N / q_cap
    int ericksen;
};

// Control block on the device.
struct Ctl {
    long long t;                 // step counter
    unsigned int ticket;         // CTA arrival counter of the node kernel
    int err_nonfinite;
    int err_body;
    int err_cfl;
    int err_timeout;             // a bounded wait of a lattice kernel gave up
    unsigned int tile_ticket;    // tile arrivals of a lattice kernel with the node tail (readout steps)
};

// Node kernel geometry: NB owned nodes per CTA, NODE_THREADS >= NB + 4 threads.
constexpr int NB = 60;
constexpr int NODE_PARTIALS = 10;
constexpr int NODE_THREADS = 64;

struct NodeArgs {
    int n_rings;
    RingDev* rings;
    int n_ctas;                  // node-kernel CTAs (>= 1)
    const int2* work;            // per CTA: (ring or -1, first owned node)
    const int* ring_cta0;        // per ring: first CTA, number of CTAs
    const int* ring_ctas;
    unsigned* ring_tickets;      // per ring: arrival counter
    double* node_partials;       // per CTA (NODE_PARTIALS): F_rest (2), COM (2), box min/max (4),
                                 // COM of the advanced positions (2)
    const double2* X;            // FP64 master node positions, wrapped into [0, n) (read)
    double2* X_out;              // the advanced positions (written; a different buffer than X when
                                 // advancing: other CTAs read their halo nodes from X meanwhile)
    int2* node_cell;
    float2* node_frac;
    float2* node_force;
    const float* ubox;
    const float* fpbox;
    const double* partials;
    int n_partials;
    double* series;              // [cap][row_len]
    int series_cap, row_len;
    Ctl* ctl;
    int every;
    int nx, ny;
    int walls_y;                 // 1: walls in y; a node closer than 4 cells to one is an error
    int walls_x;                 // 1: walls in x; the same
    int advance;                 // 0: forces + box only (initial configuration); else the steps
                                 // the positions advance by (1; 15 for a learned jump, the
                                 // velocities on the boxes then carry that factor)
};

struct FusedArgs {
    const void* src;             // state at t (N_PLANES planes: FP32, or FP16/BF16 in the precision form)
    void* dst;                   // state at t + 1
    int prec;                    // 0: FP32 state, 1: FP16 populations + BF16 sigma, dP
    int scalar;                  // 1: the scalar model (constant modulus, no P field; FP32 only)
    int walls_y;                 // 1: half-way bounce-back walls at y = -1/2, ny - 1/2 (one-cell tiles, FP32)
    int walls_x;                 // 1: the same at x = -1/2, nx - 1/2
    long long plane;             // nx * ny
    int nx, ny;
    Phys ph;
    const float2* lut;           // LUT_N + 1 entries (a2, a4)
    int n_rings;
    const RingDev* rings;
    const int2* node_cell;       // grid view of the nodes: cell, fraction, force (FP32)
    const float2* node_frac;
    const float2* node_force;
    float* ubox;                 // u(t) on each ring's box (written)
    float* fpbox;                // f^p(t) on each ring's box (written on readout steps)
    double* partials;            // per-CTA readout sums (5 per CTA)
    Ctl* ctl;
    int every;                   // readout period
    float* moments_out;          // MOMENTS mode: drho, ux, uy planes
    float* forces_out;           // MOMENTS mode, optional: Fx, Fy planes (total lattice force)
    // STEP mode with node_tail = 1: the node step of the same time step runs in the kernel's
    // tail.  Every tile whose staged region meets a ring's work box counts itself in
    // box_tickets[ring] once its u (and f^p) box writes are out; the last of them opens the
    // ring's node blocks (na, as the node kernel would run them) in ring_claim, and every tile
    // that finishes later claims and runs open blocks one at a time.  Only the tiles that meet
    // the box of step t read a ring's nodes, and the node update writes the box of step t + 1,
    // so the update needs no second launch.  The step index comes from the host (t), and
    // ctl->t is advanced during the launch.
    int node_tail;
    int tile_rot;                // node_tail: the launch order starts at this tile row, so that
                                 // the tiles over the first ring run early
    long long t;                 // node_tail: the step index
    unsigned* box_tickets;       // node_tail, per ring: arrivals of the tiles meeting its box
    unsigned long long* ring_claim;   // node_tail, per ring: (t + 1) << 16 | blocks claimed
    NodeArgs na;                 // node step of this time step (node_tail)
};

// Per-device one-time set-up (a function's shared-memory opt-in applies to one device only):
// returns false the first time it is called for the current device with this flag word, and
// marks the device; up to 64 devices.  Not thread-safe, like the handles that call it.
inline bool done_on_device(unsigned long long& flags)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
    const unsigned long long bit = 1ull << dev;
    if (flags & bit) return true;
    flags |= bit;
    return false;
}

// Launchers (return cudaError_t of the launch).
// pair: the tile kernel with two cells per thread (paired FP32 instructions)
cudaError_t launch_fused(const FusedArgs& a, int mode, cudaStream_t s, int* grid_ctas, bool pdl = false,
                         bool pair = false);
// column-strip sweep (lb_sweep.cu): eligibility, rows per CTA chunk, CTA count, launch
bool sweep_eligible(int nx, int ny);
int sweep_chunk(int nx, int ny, int n_sm);
int sweep_ctas(int nx, int ny, int chunk);
cudaError_t launch_sweep(const FusedArgs& a, int chunk, cudaStream_t s);
cudaError_t launch_nodes(const NodeArgs& a, cudaStream_t s, bool pdl = false);
// warp-strip kernel (lb_strip.cu): eligibility (walls: any wall), rows per warp chunk, CTA count,
// launch (FusedArgs::t carries the step index)
bool strip_eligible(int nx, int ny, int walls);
bool strip_preferred(int nx, int ny, int n_sm);      // faster than the tile kernel (measured)
int strip_chunk(int nx, int ny, int n_sm);
int strip_ctas(int nx, int ny, int chunk);
cudaError_t launch_strip(const FusedArgs& a, int chunk, cudaStream_t s, bool pdl);
int fused_ctas(int nx, int ny);
// the tile row holding the cell row y_top (any real value; wrapped): where the launch order of
// the tile kernel with the node tail starts
int fused_tile_rot(int nx, int ny, double y_top);

enum { MODE_STEP = 0, MODE_MOMENTS = 1 };

// Stress-diffusion sub-steps (lb_diffuse.cu): s Heun sub-steps of D_p/s on the sigma planes of
// sig_new (3 planes of NP), using sig_tmp (3 planes) as the other buffer.
int diffuse_smem_floats();
int diffuse_tiles_x(int nx);
int diffuse_tiles_y(int ny);
cudaError_t launch_diffusion(float* sig_new, float* sig_tmp, long long NP, int nx, int ny, float D, int substeps,
                             cudaStream_t s);

// Host-side table builder (FP64): fills lut[2*(LUT_N+1)] with (a2, a4) pairs.
void build_lut(double P_cap, float* lut);

}  // namespace vlb
