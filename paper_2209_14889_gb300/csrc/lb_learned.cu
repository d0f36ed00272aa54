// lb_learned.cu -- the learned stepper: the U-Net of lb_unet.cu advances (u, sigma^p, P) by 16
// lattice steps per call, checked against the plain solver and replaced by it when it fails.
//
// Field channels of the network (NHWC, 16 channels): 0 ux, 1 uy, 2 sigma_xx, 3 sigma_xy,
// 4 sigma_yy, 5 dP_x, 6 dP_y (dP = P - P_ref, the stored orientation), 7 body indicator
// (sum over ring nodes of phi(x - X_a) phi(y - Y_a), the IB kernel weights), 8..15 zero.
// Inputs are x_c = (f_c - shift_c) scale_c; the output is the change over 16 steps of channels
// 0..6 in units 1 / oscale_c.
//
// One call at step t:
//   1. moments and body indicator at t; pack x (BF16) and the raw fields f(t) (FP32);
//   2. network forward: f_net(t+16) = f(t) + y / oscale;
//   3. one plain step (t -> t+1) and its tendency T_1 = f(t+1) - f(t);
//   4. residual check: (i) momentum balance |sum u_net - sum u(t) - 16 F_pull| / (16 |F_pull|)
//      (the lattice force sums to the pull: elastic forces cancel, the stress divergences
//      telescope); (ii) tendency mismatch |(f_net - f(t))/16 - T_1| / |T_1| of sigma and P in the
//      scaled channel norm.  Both at most their epsilon: accept (the network's velocity then gets
//      the uniform correction that makes (i) exact); else run the remaining 15 plain steps.
//   5. accept: sigma and dP from the net; ring nodes advanced by 15 steps with the mean of
//      u(t+1) and u_net (one Heun step of the node kernel with 15x velocities on the work boxes);
//      populations rebuilt as the equilibrium at rho(t+1) and the velocity u_net - F/(2 rho) (the
//      network's u includes the Guo half force; F is the total force at the new state) plus the
//      regularised non-equilibrium part of a BGK fluid with the gradient of u_net,
//      f^neq_n = (9/2) w_n Q_n : Pi, Pi = -(rho tau / 3)(grad u + grad u^T), Q_n = c_n c_n - I/3.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "lb_handle.h"

using bf16 = __nv_bfloat16;

struct LearnNorm {
    float shift[8], scale[8], oscale[7];
};

namespace vlb {
namespace learn {

__device__ __forceinline__ int wrap(int i, int n)
{
    i %= n;
    return i < 0 ? i + n : i;
}
__device__ __forceinline__ double mimg(double d, double L)
{
    d -= L * floor(d / L + 0.5);
    return d;
}
__device__ __forceinline__ float phi(float r)
{
    return fabsf(r) < 2.f ? 0.25f * (1.f + cospif(0.5f * r)) : 0.f;
}

// raw fields f(t) [P][8] (channel 7: body indicator) from the state, the moment planes and the
// ring nodes; x = BF16 normalised input [P][16] (batch slot offset applied by the caller)
__global__ void k_pack(const float* st, const float* mom, long long NP, int nx, int ny, const RingDev* rings,
                       int n_rings, const double2* X, LearnNorm nm, float* raw, bf16* x, long long t)
{
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= NP) return;
    const int cx = (int)(g % nx), cy = (int)(g / nx);
    float f[8];
    f[0] = mom[NP + g];
    f[1] = mom[2 * NP + g];
    f[2] = st[PL_SXX * NP + g];
    f[3] = st[PL_SXY * NP + g];
    f[4] = st[PL_SYY * NP + g];
    f[5] = st[PL_PX * NP + g];
    f[6] = st[PL_PY * NP + g];
    float ind = 0.f;
    for (int r = 0; r < n_rings; ++r) {
        const RingDev R = rings[r];
        const int4 B = ring_box(R, t);
        const int bx = wrap(cx - B.x, nx), by = wrap(cy - B.y, ny);
        if (bx >= B.z || by >= B.w) continue;
        for (int k = 0; k < R.n_nodes; ++k) {
            const double2 p = X[R.node_off + k];
            const float dx = (float)mimg((double)cx - p.x, nx), dy = (float)mimg((double)cy - p.y, ny);
            if (fabsf(dx) < 2.f && fabsf(dy) < 2.f) ind += phi(dx) * phi(dy);
        }
    }
    f[7] = ind;
    for (int c = 0; c < 8; ++c) raw[g * 8 + c] = f[c];
    if (x) {
        __nv_bfloat162* xo = reinterpret_cast<__nv_bfloat162*>(x + g * 16);
        for (int c = 0; c < 8; c += 2)
            xo[c / 2] = __floats2bfloat162_rn((f[c] - nm.shift[c]) * nm.scale[c], (f[c + 1] - nm.shift[c + 1]) * nm.scale[c + 1]);
        for (int c = 8; c < 16; c += 2) xo[c / 2] = __floats2bfloat162_rn(0.f, 0.f);
    }
}

// residual sums (FP64, per block): 0,1 sum u_net; 2,3 sum u(t); 4 sum_c s_c^2 (T_net - T_1)^2;
// 5 sum_c s_c^2 T_1^2 over the slow fields c = 2..6 (sigma, dP) with T_net = y_c / oscale_c / 16,
// T_1 = f(t+1) - f(t), s_c = scale_c.  The velocity is left out of (ii): its change in one step
// is dominated by sound waves that a 16-step average does not follow.
__global__ void k_residual(const float* raw0, const float* y, const float* st1, const float* mom1, long long NP,
                           LearnNorm nm, double* part)
{
    __shared__ double red[6][256];
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < NP; g += (long long)gridDim.x * blockDim.x) {
        float f1[7];
        f1[0] = mom1[NP + g];
        f1[1] = mom1[2 * NP + g];
        f1[2] = st1[PL_SXX * NP + g];
        f1[3] = st1[PL_SXY * NP + g];
        f1[4] = st1[PL_SYY * NP + g];
        f1[5] = st1[PL_PX * NP + g];
        f1[6] = st1[PL_PY * NP + g];
        for (int c = 0; c < 7; ++c) {
            const float d = y[g * 16 + c] / nm.oscale[c];
            const float f0 = raw0[g * 8 + c];
            if (c < 2) {
                acc[c] += (double)(f0 + d);
                acc[2 + c] += (double)f0;
            }
            if (c >= 2) {            // the slow fields: sigma and P
                const double tn = (double)d / 16.0, t1 = (double)f1[c] - (double)f0;
                const double s2 = (double)nm.scale[c] * nm.scale[c];
                acc[4] += s2 * (tn - t1) * (tn - t1);
                acc[5] += s2 * t1 * t1;
            }
        }
    }
    for (int k = 0; k < 6; ++k) red[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int k = 0; k < 6; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 6; ++k) part[blockIdx.x * 6 + k] = red[k][0];
}

// accepted call: sigma, dP from the net into the state; u_net into unet [2][NP]; 15-step node
// velocities 7.5 (u(t+1) + u_net) on every ring's work box
__global__ void k_unpack(const float* raw0, const float* y, float* st, const float* mom, float* unet, long long NP,
                         int nx, int ny, LearnNorm nm, const RingDev* rings, int n_rings, float* ubox, float dux,
                         float duy, long long t)
{
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= NP) return;
    float f[7];
    for (int c = 0; c < 7; ++c) f[c] = raw0[g * 8 + c] + y[g * 16 + c] / nm.oscale[c];
    f[0] += dux;                 // uniform correction: the momentum balance holds exactly
    f[1] += duy;
    const float u1x = mom[NP + g], u1y = mom[2 * NP + g];
    st[PL_SXX * NP + g] = f[2];
    st[PL_SXY * NP + g] = f[3];
    st[PL_SYY * NP + g] = f[4];
    st[PL_PX * NP + g] = f[5];
    st[PL_PY * NP + g] = f[6];
    unet[g] = f[0];
    unet[NP + g] = f[1];
    const int cx = (int)(g % nx), cy = (int)(g / nx);
    for (int r = 0; r < n_rings; ++r) {
        const RingDev R = rings[r];
        const int4 B = ring_box(R, t);
        const int bx = wrap(cx - B.x, nx), by = wrap(cy - B.y, ny);
        if (bx < B.z && by < B.w) {
            const long long o = R.box_off + (long long)by * R.cap_w + bx;
            const long long cap = (long long)R.cap_w * R.cap_h;
            ubox[o] = 7.5f * (u1x + f[0]);
            ubox[o + cap] = 7.5f * (u1y + f[1]);
        }
    }
}

// populations (shifted, d_n = h_n - w_n rho0) rebuilt from drho (moment plane 0), the network's
// velocity unet and the total force F at the new state: the velocity u = (sum c h + F/2) / rho
// is the network's, so the populations carry the momentum rho u - F/2
__global__ void k_rebuild_pops(const float* mom, const float* unet, const float* frc, float* st, long long NP, int nx,
                               int ny, float rho0, float tau)
{
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= NP) return;
    const int x = (int)(g % nx), y = (int)(g / nx);
    const long long ge = (long long)y * nx + wrap(x + 1, nx), gw = (long long)y * nx + wrap(x - 1, nx);
    const long long gn = (long long)wrap(y + 1, ny) * nx + x, gs = (long long)wrap(y - 1, ny) * nx + x;
    const float* ux = unet;
    const float* uy = unet + NP;
    const float drho = mom[g];
    const float rho = rho0 + drho;
    const float u = ux[g] - 0.5f * frc[g] / rho, v = uy[g] - 0.5f * frc[NP + g] / rho;
    const float dxu = 0.5f * (ux[ge] - ux[gw]), dyu = 0.5f * (ux[gn] - ux[gs]);
    const float dxv = 0.5f * (uy[ge] - uy[gw]), dyv = 0.5f * (uy[gn] - uy[gs]);
    const float k = -rho * tau / 3.f;
    const float Pxx = k * 2.f * dxu, Pyy = k * 2.f * dyv, Pxy = k * (dyu + dxv);
    const float trP = Pxx + Pyy;
    const int cxs[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    const int cys[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    const float ws[9] = {4.f / 9.f, 1.f / 9.f, 1.f / 9.f, 1.f / 9.f, 1.f / 9.f, 1.f / 36.f, 1.f / 36.f, 1.f / 36.f, 1.f / 36.f};
    const float uu = u * u + v * v;
    for (int n = 0; n < 9; ++n) {
        const float cx = (float)cxs[n], cy = (float)cys[n];
        const float cu = cx * u + cy * v;
        const float eq = ws[n] * (drho + rho * (3.f * cu + 4.5f * cu * cu - 1.5f * uu));
        const float QP = cx * cx * Pxx + 2.f * cx * cy * Pxy + cy * cy * Pyy - trP / 3.f;
        st[n * NP + g] = eq + 4.5f * ws[n] * QP;
    }
}

// network input from raw fields: x_c = (f_c - shift_c) scale_c for c < 8, zero above
__global__ void k_normalize(const float* raw, LearnNorm nm, long long P, bf16* x)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P * 16) return;
    const long long g = i / 16;
    const int c = (int)(i - g * 16);
    x[i] = __float2bfloat16_rn(c < 8 ? (raw[g * 8 + c] - nm.shift[c]) * nm.scale[c] : 0.f);
}

// training target: the change of channels 0..6 over the pair, in output units; 7..15 zero
__global__ void k_target(const float* raw0, const float* raw1, LearnNorm nm, long long P, float* target)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P * 16) return;
    const long long g = i / 16;
    const int c = (int)(i - g * 16);
    target[i] = c < 7 ? (raw1[g * 8 + c] - raw0[g * 8 + c]) * nm.oscale[c] : 0.f;
}

}  // namespace learn
}  // namespace vlb

using namespace vlb;
using namespace vlb::learn;

struct lb_learned {
    lb_handle* h = nullptr;
    lb_net* net = nullptr;
    LearnNorm nm;
    double eps_mom = 0.0, eps_tend = 0.0;
    float* raw0 = nullptr;       // [P][8]
    float* unet = nullptr;       // [2][P] the network's velocity of an accepted call
    float* frc = nullptr;        // [2][P] total lattice force at the new state
    bf16* x = nullptr;           // [P][16]
    double* part = nullptr;      // residual partials
    int nb = 0;
    double fpull_x = 0.0, fpull_y = 0.0;
    double last[2] = {0.0, 0.0};
    long long calls = 0, accepted = 0;
    std::string err;
};

namespace {

int lfail(lb_learned* L, int code, const std::string& m)
{
    if (L) L->err = m;
    return code;
}

#define LCK(L, call)                                                                   \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            if (L) L->err = std::string(#call) + ": " + cudaGetErrorString(e_);        \
            return LB_ECUDA;                                                           \
        }                                                                              \
    } while (0)

int blocks(long long n) { return (int)((n + 255) / 256); }

// moments of the handle's current state into h->moments (allocated on first use), and the total
// lattice force into frc [2][NP] when given
int moments(lb_handle* h, float* frc = nullptr)
{
    if (!h->moments && cudaMalloc(&h->moments, sizeof(float) * 3 * (size_t)h->plane) != cudaSuccess) return LB_ENOMEM;
    FusedArgs fa = handle_fused_args(h);
    fa.moments_out = h->moments;
    fa.forces_out = frc;
    return launch_fused(fa, MODE_MOMENTS, h->stream, nullptr) == cudaSuccess ? LB_OK : LB_ECUDA;
}

int pack(lb_handle* h, const LearnNorm& nm, float* raw, bf16* x)
{
    int rc = moments(h);
    if (rc != LB_OK) return rc;
    k_pack<<<blocks(h->plane), 256, 0, h->stream>>>(static_cast<const float*>(h->state[h->cur]), h->moments, h->plane,
                                                    h->p.nx, h->p.ny, h->rings, h->n_rings, h->X, nm, raw, x, h->t);
    return cudaGetLastError() == cudaSuccess ? LB_OK : LB_ECUDA;
}

bool read_norm(const float* norm, LearnNorm& nm)
{
    for (int c = 0; c < 8; ++c) {
        nm.shift[c] = norm[c];
        nm.scale[c] = norm[8 + c];
    }
    for (int c = 0; c < 7; ++c) nm.oscale[c] = norm[16 + c];
    for (int c = 0; c < 8; ++c)
        if (!std::isfinite(nm.shift[c]) || !std::isfinite(nm.scale[c])) return false;
    for (int c = 0; c < 7; ++c)
        if (!(nm.oscale[c] > 0.f) || !std::isfinite(nm.oscale[c])) return false;
    return true;
}

}  // namespace

extern "C" {

int lb_learned_pack(lb_handle* h, const float* norm, void* x, float* raw)
{
    if (!h || !norm || (!x && !raw)) return LB_EINVAL;
    if (!h->fields_ready) return LB_ESTATE;
    if (h->p.precision != LB_FP32) return LB_EINVAL;
    LearnNorm nm;
    if (!read_norm(norm, nm)) return LB_EINVAL;
    float* r = raw;
    float* tmp = nullptr;
    if (!r) {
        if (cudaMalloc(&tmp, sizeof(float) * 8 * (size_t)h->plane) != cudaSuccess) return LB_ENOMEM;
        r = tmp;
    }
    const int rc = pack(h, nm, r, static_cast<bf16*>(x));
    if (tmp) {
        cudaStreamSynchronize(h->stream);
        cudaFree(tmp);
    }
    return rc;
}

int lb_learned_target(const float* raw0, const float* raw1, const float* norm, float* target, int64_t cells,
                      void* stream)
{
    if (!raw0 || !raw1 || !norm || !target || cells < 1) return LB_EINVAL;
    LearnNorm nm;
    if (!read_norm(norm, nm)) return LB_EINVAL;
    k_target<<<blocks(cells * 16), 256, 0, (cudaStream_t)stream>>>(raw0, raw1, nm, cells, target);
    return cudaGetLastError() == cudaSuccess ? LB_OK : LB_ECUDA;
}

int lb_learned_normalize(const float* raw, const float* norm, void* x, int64_t cells, void* stream)
{
    if (!raw || !norm || !x || cells < 1) return LB_EINVAL;
    LearnNorm nm;
    if (!read_norm(norm, nm)) return LB_EINVAL;
    k_normalize<<<blocks(cells * 16), 256, 0, (cudaStream_t)stream>>>(raw, nm, cells, static_cast<bf16*>(x));
    return cudaGetLastError() == cudaSuccess ? LB_OK : LB_ECUDA;
}

int lb_learned_create(lb_handle* h, lb_net* net, const float* norm, double eps_momentum, double eps_tendency,
                      lb_learned** out)
{
    if (!h || !net || !norm || !out) return LB_EINVAL;
    *out = nullptr;
    if (!h->fields_ready || !h->node_work) return LB_ESTATE;
    if (h->p.precision != LB_FP32 || h->p.model != LB_MODEL_TENSORIAL || h->p.walls_y || h->p.walls_x || h->p.readout_every % 16 != 0)
        return LB_EINVAL;
    int32_t nb = 0, nh = 0, nw = 0;
    if (lb_net_shape(net, &nb, &nh, &nw) != LB_OK || nb != 1 || nh != h->p.ny || nw != h->p.nx) return LB_EINVAL;
    lb_learned* L = new lb_learned();
    L->h = h;
    L->net = net;
    if (!read_norm(norm, L->nm) || !(eps_momentum > 0.0) || !(eps_tendency > 0.0)) {
        delete L;
        return LB_EINVAL;
    }
    L->eps_mom = eps_momentum;
    L->eps_tend = eps_tendency;
    L->nb = 148;
    if (cudaMalloc(&L->raw0, sizeof(float) * 8 * (size_t)h->plane) != cudaSuccess ||
        cudaMalloc(&L->unet, sizeof(float) * 2 * (size_t)h->plane) != cudaSuccess ||
        cudaMalloc(&L->frc, sizeof(float) * 2 * (size_t)h->plane) != cudaSuccess ||
        cudaMalloc(&L->x, sizeof(bf16) * 16 * (size_t)h->plane) != cudaSuccess ||
        cudaMalloc(&L->part, sizeof(double) * 6 * L->nb) != cudaSuccess) {
        lb_learned_destroy(L);
        return LB_ENOMEM;
    }
    // total pull force on the rings: the sum of the lattice force
    if (h->n_rings > 0) {
        std::vector<RingDev> rd(h->n_rings);
        if (cudaMemcpy(rd.data(), h->rings, sizeof(RingDev) * h->n_rings, cudaMemcpyDeviceToHost) != cudaSuccess) {
            lb_learned_destroy(L);
            return LB_ECUDA;
        }
        for (const RingDev& r : rd) {
            L->fpull_x += r.pull_x * r.n_nodes;
            L->fpull_y += r.pull_y * r.n_nodes;
        }
    }
    *out = L;
    return LB_OK;
}

int lb_learned_step(lb_learned* L, int64_t calls, int64_t* n_fallbacks)
{
    if (!L || calls < 0) return LB_EINVAL;
    lb_handle* h = L->h;
    int64_t fb = 0;
    const double F = std::sqrt(L->fpull_x * L->fpull_x + L->fpull_y * L->fpull_y);
    std::vector<double> part(6 * L->nb);
    for (int64_t k = 0; k < calls; ++k) {
        int rc = pack(h, L->nm, L->raw0, L->x);
        if (rc != LB_OK) return lfail(L, rc, "pack");
        rc = lb_net_forward(L->net, L->x, nullptr);
        if (rc != LB_OK) return lfail(L, rc, std::string("network: ") + lb_net_last_error(L->net));
        const float* y = lb_net_output(L->net);
        rc = lb_step(h, 1);
        if (rc != LB_OK) return lfail(L, rc, lb_last_error(h));
        rc = moments(h);
        if (rc != LB_OK) return lfail(L, rc, "moments");
        k_residual<<<L->nb, 256, 0, h->stream>>>(L->raw0, y, static_cast<const float*>(h->state[h->cur]), h->moments,
                                                 h->plane, L->nm, L->part);
        LCK(L, cudaGetLastError());
        LCK(L, cudaMemcpyAsync(part.data(), L->part, sizeof(double) * 6 * L->nb, cudaMemcpyDeviceToHost, h->stream));
        LCK(L, cudaStreamSynchronize(h->stream));
        double s[6] = {0, 0, 0, 0, 0, 0};
        for (int b = 0; b < L->nb; ++b)
            for (int c = 0; c < 6; ++c) s[c] += part[b * 6 + c];
        const double mx = s[0] - s[2] - 16.0 * L->fpull_x, my = s[1] - s[3] - 16.0 * L->fpull_y;
        const double r_mom = std::sqrt(mx * mx + my * my) / (16.0 * F > 0.0 ? 16.0 * F : 1e-30);
        const double r_tend = std::sqrt(s[4] / (s[5] > 0.0 ? s[5] : 1e-300));
        L->last[0] = r_mom;
        L->last[1] = r_tend;
        L->calls += 1;
        const bool ok = std::isfinite(r_mom) && std::isfinite(r_tend) && r_mom <= L->eps_mom && r_tend <= L->eps_tend;
        if (!ok) {
            rc = lb_step(h, 15);
            if (rc != LB_OK) return lfail(L, rc, lb_last_error(h));
            ++fb;
            continue;
        }
        L->accepted += 1;
        // sigma, dP and the node jump first; then the force at the new state (the moments
        // pass reads the populations of t+1, unchanged, for drho); then the populations
        float* st = static_cast<float*>(h->state[h->cur]);
        // uniform velocity correction so that sum u_net = sum u(t) + 16 F_pull exactly
        const float dux = (float)(-mx / (double)h->plane), duy = (float)(-my / (double)h->plane);
        k_unpack<<<blocks(h->plane), 256, 0, h->stream>>>(L->raw0, y, st, h->moments, L->unet, h->plane, h->p.nx,
                                                          h->p.ny, L->nm, h->rings, h->n_rings, h->ubox, dux, duy,
                                                          h->t);
        LCK(L, cudaGetLastError());
        LCK(L, launch_nodes(handle_node_args(h, 15), h->stream, false));
        std::swap(h->X, h->X_alt);
        h->t += 15;
        rc = moments(h, L->frc);
        if (rc != LB_OK) return lfail(L, rc, "moments");
        k_rebuild_pops<<<blocks(h->plane), 256, 0, h->stream>>>(h->moments, L->unet, L->frc, st, h->plane, h->p.nx,
                                                                h->p.ny, (float)h->p.rho0, (float)h->p.tau);
        LCK(L, cudaGetLastError());
    }
    if (n_fallbacks) *n_fallbacks = fb;
    return LB_OK;
}

int lb_learned_stats(const lb_learned* L, double* out4)
{
    if (!L || !out4) return LB_EINVAL;
    out4[0] = L->last[0];
    out4[1] = L->last[1];
    out4[2] = (double)L->calls;
    out4[3] = (double)L->accepted;
    return LB_OK;
}

const char* lb_learned_last_error(const lb_learned* L) { return L ? L->err.c_str() : "null learned stepper"; }

void lb_learned_destroy(lb_learned* L)
{
    if (!L) return;
    if (L->h && L->h->stream) cudaStreamSynchronize(L->h->stream);
    cudaFree(L->raw0);
    cudaFree(L->unet);
    cudaFree(L->frc);
    cudaFree(L->x);
    cudaFree(L->part);
    delete L;
}

}  // extern "C"
