// lb_api.cu -- the C ABI declared in include/lb.h: handle, validation, device buffers, launches.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "lb_handle.h"

using namespace vlb;


namespace {

std::string g_err;

int fail(lb_handle* h, int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h) h->err = buf; else g_err = buf;
    return code;
}

int cuda_fail(lb_handle* h, cudaError_t e, const char* what)
{
    return fail(h, e == cudaErrorMemoryAllocation ? LB_ENOMEM : LB_ECUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

#define CK(h, call)                                         \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
    } while (0)

template <class T>
void dfree(T*& p)
{
    if (p) cudaFree(p);
    p = nullptr;
}

void free_rings(lb_handle* h)
{
    dfree(h->rings);
    dfree(h->X);
    dfree(h->X_alt);
    dfree(h->node_cell);
    dfree(h->node_frac);
    dfree(h->node_force);
    dfree(h->ubox);
    dfree(h->fpbox);
    dfree(h->node_work);
    dfree(h->ring_cta0);
    dfree(h->ring_ctas);
    dfree(h->ring_tickets);
    dfree(h->box_tickets);
    dfree(h->ring_claim);
    dfree(h->node_partials);
    h->n_node_ctas = 1;
    h->n_rings = h->n_total = 0;
    h->tile_rot = 0;
    h->row_len = 6;
}

cudaEvent_t ev_get(std::vector<cudaEvent_t>& pool, size_t& used)
{
    if (used == pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        pool.push_back(e);
    }
    return pool[used++];
}

FusedArgs fused_args(lb_handle* h)
{
    FusedArgs a = {};
    a.src = h->state[h->cur];
    a.dst = h->state[h->cur ^ 1];
    a.prec = h->p.precision == LB_FP32 ? 0 : 1;
    a.scalar = h->p.model == LB_MODEL_SCALAR ? 1 : 0;
    a.walls_y = h->p.walls_y;
    a.walls_x = h->p.walls_x;
    a.plane = h->plane;
    a.nx = h->p.nx;
    a.ny = h->p.ny;
    a.ph = h->ph;
    a.lut = h->lut;
    a.n_rings = h->n_rings;
    a.rings = h->rings;
    a.node_cell = h->node_cell;
    a.node_frac = h->node_frac;
    a.node_force = h->node_force;
    a.ubox = h->ubox;
    a.fpbox = h->fpbox;
    a.partials = h->partials;
    a.ctl = h->ctl;
    a.every = h->p.readout_every;
    a.moments_out = h->moments;
    a.forces_out = nullptr;
    return a;
}

// the lattice kernel of lb_step is the warp-strip kernel: chosen, or LB_KERNEL_AUTO where it
// applies and measured faster than the tile kernel
bool uses_strip(const lb_handle* h)
{
    if (h->kernel == LB_KERNEL_STRIP) return true;
    return h->kernel == LB_KERNEL_AUTO && strip_eligible(h->p.nx, h->p.ny, h->p.walls_x || h->p.walls_y) &&
           strip_preferred(h->p.nx, h->p.ny, h->n_sm);
}

NodeArgs node_args(lb_handle* h, int advance)
{
    NodeArgs a;
    a.n_rings = h->n_rings;
    a.rings = h->rings;
    a.X = h->X;
    a.X_out = advance ? h->X_alt : h->X;     // no advance: the same values written in place
    a.node_cell = h->node_cell;
    a.node_frac = h->node_frac;
    a.node_force = h->node_force;
    a.ubox = h->ubox;
    a.fpbox = h->fpbox;
    a.partials = h->partials;
    a.n_partials = h->n_partials;
    a.series = h->series;
    a.series_cap = h->series_cap;
    a.row_len = h->row_len;
    a.ctl = h->ctl;
    a.every = h->p.readout_every;
    a.nx = h->p.nx;
    a.ny = h->p.ny;
    a.walls_y = h->p.walls_y;
    a.walls_x = h->p.walls_x;
    a.advance = advance;
    a.n_ctas = h->n_node_ctas;
    a.work = h->node_work;
    a.ring_cta0 = h->ring_cta0;
    a.ring_ctas = h->ring_ctas;
    a.ring_tickets = h->ring_tickets;
    a.node_partials = h->node_partials;
    return a;
}

// The C~ table depends only on P_cap; it is built once per value in the process.
void cached_lut(double P_cap, std::vector<float>& out)
{
    static std::mutex mu;
    static std::map<double, std::vector<float>> cache;
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(P_cap);
    if (it == cache.end()) {
        std::vector<float> t(2 * (LUT_N + 1));
        build_lut(P_cap, t.data());
        it = cache.emplace(P_cap, std::move(t)).first;
    }
    out = it->second;
}

// Plane conversions between the stored form and FP32 values: v = stored * scale + shift.
// kind 0: FP32 plane, 1: FP16 plane (scaled populations), 2: BF16 plane.
__global__ void k_plane_to_f32(float* dst, const void* src, int kind, float scale, float shift, long long n)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float v;
    if (kind == 0) v = static_cast<const float*>(src)[i];
    else if (kind == 1) v = __half2float(static_cast<const __half*>(src)[i]);
    else v = __bfloat162float(static_cast<const __nv_bfloat16*>(src)[i]);
    dst[i] = v * scale + shift;
}

// stored = (v - shift) * scale, round to nearest (initial and user-written fields)
__global__ void k_f32_to_plane(void* dst, const float* src, int kind, float scale, float shift, long long n)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float v = (src[i] - shift) * scale;
    if (kind == 0) static_cast<float*>(dst)[i] = v;
    else if (kind == 1) static_cast<__half*>(dst)[i] = __float2half_rn(v);
    else static_cast<__nv_bfloat16*>(dst)[i] = __float2bfloat16_rn(v);
}

// stored plane p of buffer b: base pointer, kind, and the (scale, shift) that maps it to the
// physical value (populations: d_n; sigma; P = dP + P_ref)
struct PlaneInfo {
    void* ptr;
    int kind;
    float scale, shift;
};

PlaneInfo plane_info(const lb_handle* h, int b, int plane)
{
    PlaneInfo pi;
    const size_t N = (size_t)h->plane;
    pi.ptr = static_cast<char*>(h->state[b]) + (size_t)h->esz * plane * N;
    const bool lp = h->p.precision != LB_FP32;
    pi.kind = !lp ? 0 : ((plane < PL_SXX || plane >= PL_PX) ? 1 : 2);   // FP16 pops and dP, BF16 sigma
    pi.scale = 1.f;
    pi.shift = 0.f;
    if (lp && plane < PL_SXX) {
        const double w = plane == 0 ? 4.0 / 9.0 : (plane < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
        pi.scale = (float)(w / 4096.0);       // stored s_n = d_n 2^12 / w_n
    }
    if (plane == PL_PX) pi.shift = h->ph.prx;
    if (plane == PL_PY) pi.shift = h->ph.pry;
    return pi;
}

cudaError_t plane_to_f32(const lb_handle* h, int b, int plane, float* dst)
{
    const PlaneInfo pi = plane_info(h, b, plane);
    const long long n = h->plane;
    k_plane_to_f32<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(dst, pi.ptr, pi.kind, pi.scale, pi.shift, n);
    return cudaGetLastError();
}

cudaError_t f32_to_plane(const lb_handle* h, int b, int plane, const float* src)
{
    const PlaneInfo pi = plane_info(h, b, plane);
    const long long n = h->plane;
    k_f32_to_plane<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(pi.ptr, src, pi.kind, 1.f / pi.scale,
                                                                      pi.shift, n);
    return cudaGetLastError();
}

}  // namespace

namespace vlb {
FusedArgs handle_fused_args(lb_handle* h) { return fused_args(h); }
NodeArgs handle_node_args(lb_handle* h, int advance) { return node_args(h, advance); }
}  // namespace vlb

extern "C" {

int lb_create(const lb_params* pin, void* stream, lb_handle** out)
{
    if (!pin || !out) return fail(nullptr, LB_EINVAL, "null argument");
    *out = nullptr;
    const lb_params& p = *pin;
    if (p.nx < 8 || p.ny < 8) return fail(nullptr, LB_EINVAL, "nx, ny must be >= 8");
    if ((long long)p.nx * p.ny > (1LL << 31)) return fail(nullptr, LB_EINVAL, "lattice too large");
    if (p.precision != LB_FP32 && p.precision != LB_FP16_BF16)
        return fail(nullptr, LB_EINVAL, "unsupported precision %d", p.precision);
    if (!(p.tau > 0.5) || !(p.rho0 > 0.0)) return fail(nullptr, LB_EINVAL, "need tau > 1/2, rho0 > 0");
    if (!(p.P_cap > 0.0 && p.P_cap < 1.0)) return fail(nullptr, LB_EINVAL, "need 0 < P_cap < 1");
    if (p.readout_every < 1 || p.max_samples < 1) return fail(nullptr, LB_EINVAL, "bad readout settings");
    const double S8 = (3 * p.K1111 + 2 * p.K1122 + 4 * p.K1212 + 3 * p.K2222) / 8.0;
    double eta = p.eta_p;
    if (!(eta > 0.0)) eta = p.lambda_steps * S8;
    if (!(eta > 0.0) || !std::isfinite(eta)) return fail(nullptr, LB_EINVAL, "need eta_p > 0 or lambda_steps > 0");
    // explicit stability bounds of the Heun steps (|z| <= 2 on the negative real axis)
    if (p.model != LB_MODEL_TENSORIAL && p.model != LB_MODEL_SCALAR)
        return fail(nullptr, LB_EINVAL, "unknown model %d", p.model);
    if (p.model == LB_MODEL_SCALAR) {
        if (p.precision != LB_FP32) return fail(nullptr, LB_EINVAL, "the scalar model needs the FP32 state");
        if (p.ericksen) return fail(nullptr, LB_EINVAL, "the scalar model has no Ericksen force (ericksen = 0)");
        const double C = p.K1111, tol = 1e-12 * std::fabs(C);
        if (!(C > 0.0) || std::fabs(p.K2222 - C) > tol || std::fabs(p.K1122) > tol || std::fabs(p.K1212 - 0.5 * C) > tol)
            return fail(nullptr, LB_EINVAL, "the scalar model needs K2222 = K1111, K1122 = 0, K1212 = K1111 / 2");
    }
    if (p.walls_y != 0 && p.walls_y != 1) return fail(nullptr, LB_EINVAL, "walls_y must be 0 or 1");
    if (p.walls_x != 0 && p.walls_x != 1) return fail(nullptr, LB_EINVAL, "walls_x must be 0 or 1");
    // a ghost cell is then at most one mirror away from its image (a negated image is negated once)
    if ((p.walls_y && p.ny < 4) || (p.walls_x && p.nx < 4))
        return fail(nullptr, LB_EINVAL, "a walled axis needs at least 4 cells");
    if ((p.walls_y || p.walls_x) && (p.precision != LB_FP32 || p.diffusion_substeps != 0))
        return fail(nullptr, LB_EINVAL, "walls need the FP32 state and no diffusion sub-steps");
    if (p.diffusion_substeps < 0) return fail(nullptr, LB_EINVAL, "diffusion_substeps < 0");
    if (p.diffusion_substeps > 0 && p.precision != LB_FP32)
        return fail(nullptr, LB_EINVAL, "diffusion sub-steps need the FP32 state");
    const int dsub = p.diffusion_substeps;
    if (p.Dp < 0.0 || 8.0 * p.Dp / (dsub > 0 ? dsub : 1) > 2.0)
        return fail(nullptr, LB_EUNSTABLE, "D_p = %g with %d sub-steps outside the Heun bound 8 D_p / s <= 2",
                    p.Dp, dsub);
    const double be_rate = p.Gamma * (2.0 * std::fabs(p.alpha) + 8.0 * p.kappa);
    if (p.Gamma < 0.0 || p.kappa < 0.0 || be_rate > 2.0)
        return fail(nullptr, LB_EUNSTABLE, "Gamma (2|alpha| + 8 kappa) = %g > 2", be_rate);
    const double c_rate = (std::fabs(S8) + std::fabs(p.K1111 - p.K2222) +
                           std::fabs(p.K1111 - 2 * p.K1122 - 4 * p.K1212 + p.K2222)) / eta;
    if (c_rate > 2.0) return fail(nullptr, LB_EUNSTABLE, "stress relaxation rate %g > 2", c_rate);

    lb_handle* h = new lb_handle();
    h->p = p;
    h->stream = (cudaStream_t)stream;
    h->eta_p = eta;
    h->plane = (long long)p.nx * p.ny;
    Phys& ph = h->ph;
    ph.omega = (float)(1.0 / p.tau);
    ph.guo = (float)(1.0 - 0.5 / p.tau);
    ph.rho0 = (float)p.rho0;
    ph.alpha = (float)p.alpha;
    ph.beta = (float)p.beta;
    ph.xi = (float)p.xi;
    ph.Gamma = (float)p.Gamma;
    ph.kappa = (float)p.kappa;
    ph.Dp = p.diffusion_substeps > 0 ? 0.f : (float)p.Dp;    // sub-stepped separately
    ph.inv_eta = (float)(1.0 / eta);
    {
        const double Peq = (p.alpha < 0.0 && p.beta > 0.0) ? std::sqrt(-p.alpha / p.beta) : 0.0;
        ph.prx = (float)(Peq * std::cos(p.director_angle));
        ph.pry = (float)(Peq * std::sin(p.director_angle));
        const double rx = ph.prx, ry = ph.pry;
        ph.A0 = (float)(p.alpha + p.beta * (rx * rx + ry * ry));
    }
    ph.kS8 = (float)S8;
    ph.kC12 = (float)((p.K1111 + 6 * p.K1122 - 4 * p.K1212 + p.K2222) / 8.0);
    ph.kC33 = (float)((p.K1111 - 2 * p.K1122 + 4 * p.K1212 + p.K2222) / 4.0);
    ph.dK = (float)(p.K1111 - p.K2222);
    ph.kX = (float)(p.K1111 - 2 * p.K1122 - 4 * p.K1212 + p.K2222);
    ph.q_cap = (float)(p.P_cap * p.P_cap);
    ph.lut_scale = (float)(LUT_N / (p.P_cap * p.P_cap));
    ph.ericksen = p.ericksen ? 1 : 0;

    int rc = LB_OK;
    auto bail = [&](int code) {
        lb_destroy(h);
        return code;
    };
    h->esz = p.precision == LB_FP32 ? 4 : 2;
    const size_t state_bytes = (size_t)h->esz * N_PLANES * (size_t)h->plane;
    for (int b = 0; b < 2; ++b) {
        cudaError_t e = cudaMalloc(&h->state[b], state_bytes);
        if (e != cudaSuccess) { rc = cuda_fail(nullptr, e, "cudaMalloc(state)"); return bail(rc); }
    }
    std::vector<float> lut;
    cached_lut(p.P_cap, lut);
    int dev = 0, n_sm = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    h->sweep_chunk = sweep_chunk(p.nx, p.ny, n_sm);
    h->n_sm = n_sm;
    h->strip_chunk = strip_chunk(p.nx, p.ny, n_sm);
    h->n_partials = fused_ctas(p.nx, p.ny);
    const int partial_cap = std::max(std::max(h->n_partials, sweep_ctas(p.nx, p.ny, h->sweep_chunk)),
                                     strip_ctas(p.nx, p.ny, h->strip_chunk));
    h->partial_cap = partial_cap;
    h->series_cap = p.max_samples;
    cudaError_t e;
    if ((e = cudaMalloc(&h->lut, sizeof(float) * lut.size())) != cudaSuccess ||
        (e = cudaMalloc(&h->ctl, sizeof(Ctl))) != cudaSuccess ||
        (e = cudaMalloc(&h->partials, sizeof(double) * 5 * (size_t)partial_cap)) != cudaSuccess) {
        rc = cuda_fail(nullptr, e, "cudaMalloc");
        return bail(rc);
    }
    if ((e = cudaMemcpy(h->lut, lut.data(), sizeof(float) * lut.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(h->ctl, 0, sizeof(Ctl))) != cudaSuccess) {
        rc = cuda_fail(nullptr, e, "upload");
        return bail(rc);
    }
    if ((e = cudaMalloc(&h->series, sizeof(double) * (size_t)h->series_cap * 6)) != cudaSuccess) {
        rc = cuda_fail(nullptr, e, "cudaMalloc(series)");
        return bail(rc);
    }
    {
        const int2 w0 = make_int2(-1, 0);
        if ((e = cudaMalloc(&h->node_work, sizeof(int2))) != cudaSuccess ||
            (e = cudaMemcpy(h->node_work, &w0, sizeof(int2), cudaMemcpyHostToDevice)) != cudaSuccess ||
            (e = cudaMalloc(&h->node_partials, sizeof(double) * NODE_PARTIALS)) != cudaSuccess) {
            rc = cuda_fail(nullptr, e, "cudaMalloc(node work)");
            return bail(rc);
        }
        h->n_node_ctas = 1;
    }
    *out = h;
    return LB_OK;
}

int lb_init_fields(lb_handle* h, const double* noise)
{
    if (!h) return fail(nullptr, LB_EINVAL, "null handle");
    const lb_params& p = h->p;
    const size_t N = (size_t)h->plane;
    std::vector<float> buf(N);
    void* S = h->state[h->cur];
    // populations at rest (shifted form: zero) and sigma = 0 (zero bits in every storage form)
    CK(h, cudaMemsetAsync(S, 0, (size_t)h->esz * N_PLANES * N, h->stream));
    // stored: dP = P - P_ref with P = P_eq (cos theta_d, sin theta_d) + noise (FP64 here)
    const double Peq = (p.alpha < 0.0 && p.beta > 0.0) ? std::sqrt(-p.alpha / p.beta) : 0.0;
    float* tmp = nullptr;
    CK(h, cudaMalloc(&tmp, sizeof(float) * N));
    int rc = LB_OK;
    for (int c = 0; c < 2 && rc == LB_OK; ++c) {
        const double base = Peq * (c == 0 ? std::cos(p.director_angle) : std::sin(p.director_angle));
        const double ref = c == 0 ? h->ph.prx : h->ph.pry;
        // P itself goes through f32_to_plane, which subtracts P_ref; the deviation is formed in
        // FP64 here and P_ref added back in FP32 only where the result is exact enough
        for (size_t i = 0; i < N; ++i) buf[i] = (float)((base - ref) + (noise ? noise[c * N + i] : 0.0));
        cudaError_t e = cudaMemcpyAsync(tmp, buf.data(), sizeof(float) * N, cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) {
            // dP planes directly (no shift: buf already holds P - P_ref)
            const PlaneInfo pi = plane_info(h, h->cur, PL_PX + c);
            k_f32_to_plane<<<(unsigned)((N + 255) / 256), 256, 0, h->stream>>>(pi.ptr, tmp, pi.kind, 1.f, 0.f,
                                                                             (long long)N);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) rc = cuda_fail(h, e, "lb_init_fields");
    }
    cudaFree(tmp);
    if (rc != LB_OK) return rc;
    if (h->p.model == LB_MODEL_SCALAR) {
        // the scalar model never writes P: both buffers keep the initial field
        const size_t pb = (size_t)h->esz * N;
        CK(h, cudaMemcpyAsync(static_cast<char*>(h->state[h->cur ^ 1]) + PL_PX * pb,
                              static_cast<const char*>(h->state[h->cur]) + PL_PX * pb, 2 * pb,
                              cudaMemcpyDeviceToDevice, h->stream));
    }
    CK(h, cudaMemsetAsync(h->ctl, 0, sizeof(Ctl), h->stream));
    h->t = 0;
    h->after_tail = false;
    if (h->n_rings > 0) {
        // restart at t = 0: the work box of the current positions into the slot of even steps
        CK(h, cudaMemsetAsync(h->box_tickets, 0, sizeof(unsigned) * h->n_rings, h->stream));
        CK(h, cudaMemsetAsync(h->ring_claim, 0, sizeof(unsigned long long) * h->n_rings, h->stream));
        CK(h, launch_nodes(node_args(h, 0), h->stream));
    }
    h->fields_ready = true;
    CK(h, cudaStreamSynchronize(h->stream));
    return LB_OK;
}

int lb_set_body(lb_handle* h, int32_t n_rings, const lb_ring* rings, const double* xy)
{
    if (!h) return fail(nullptr, LB_EINVAL, "null handle");
    if (n_rings < 0 || (n_rings > 0 && (!rings || !xy))) return fail(h, LB_EINVAL, "bad rings");
    CK(h, cudaStreamSynchronize(h->stream));
    free_rings(h);
    const int nx = h->p.nx, ny = h->p.ny;
    std::vector<RingDev> rd(n_rings);
    std::vector<double2> X;
    long long box_off = 0;
    int off = 0;
    for (int r = 0; r < n_rings; ++r) {
        const lb_ring& g = rings[r];
        if (g.n_nodes < 3 || g.n_nodes > 1024) return fail(h, LB_EINVAL, "ring %d: 3 <= n_nodes <= 1024", r);
        if (!(g.l_eq > 0.0) || g.k_spring < 0.0) return fail(h, LB_EINVAL, "ring %d: bad spring", r);
        if (!(g.trap_k >= 0.0) || (g.trap_k > 0.0 && !(g.trap_width > 0.0 && g.trap_pull > 0.0 &&
                                                       std::isfinite(g.trap_dx) && std::isfinite(g.trap_dy) &&
                                                       std::isfinite(g.trap_t_eq))))
            return fail(h, LB_EINVAL, "ring %d: bad trap (k >= 0; width, pull > 0)", r);
        double mnx = 1e300, mxx = -1e300, mny = 1e300, mxy = -1e300, sdx = 0.0, sdy = 0.0;
        const double* P = xy + 2 * (size_t)off;
        for (int k = 0; k < g.n_nodes; ++k) {
            double dx = P[2 * k] - P[0], dy = P[2 * k + 1] - P[1];
            dx -= nx * std::floor(dx / nx + 0.5);
            dy -= ny * std::floor(dy / ny + 0.5);
            mnx = std::fmin(mnx, dx); mxx = std::fmax(mxx, dx);
            mny = std::fmin(mny, dy); mxy = std::fmax(mxy, dy);
            sdx += dx;
            sdy += dy;
            if (!std::isfinite(P[2 * k]) || !std::isfinite(P[2 * k + 1]))
                return fail(h, LB_EINVAL, "ring %d: non-finite node", r);
            if ((h->p.walls_y && (P[2 * k + 1] < 5.0 || P[2 * k + 1] > ny - 6.0)) ||
                (h->p.walls_x && (P[2 * k] < 5.0 || P[2 * k] > nx - 6.0)))
                return fail(h, LB_EINVAL, "ring %d: a node within 5 cells of a wall", r);
            double xw = std::fmod(P[2 * k], (double)nx); if (xw < 0) xw += nx; if (xw >= nx) xw -= nx;
            double yw = std::fmod(P[2 * k + 1], (double)ny); if (yw < 0) yw += ny; if (yw >= ny) yw -= ny;
            X.push_back(make_double2(xw, yw));
        }
        // box capacity: the initial extent + supports + a margin for motion and deformation
        // positions relative to node 0 are taken as minimum images: the ring (with the
        // supports of its nodes) must span less than half the lattice
        const int lim = std::min(nx, ny) - 8;
        int cw = (int)std::ceil(mxx - mnx) + 8, chh = (int)std::ceil(mxy - mny) + 8;
        // the tail launches start at the tile row over the first ring's top (minus the box
        // margin and the staged halo), so its node blocks run while most tiles are still to come
        if (r == 0) h->tile_rot = fused_tile_rot(nx, ny, P[1] + mny - 4.0);
        if (2 * cw > nx || 2 * chh > ny) return fail(h, LB_EINVAL, "ring %d does not fit the lattice", r);
        cw = std::min(cw + 2 * std::max(16, cw / 2), lim);
        chh = std::min(chh + 2 * std::max(16, chh / 2), lim);
        RingDev& d = rd[r];
        d.n_nodes = g.n_nodes;
        d.node_off = off;
        // the trap: protocol, initial centre of mass (node 0 plus the mean minimum-image offset,
        // wrapped), no force before the set-up pass below
        d.trap_k = g.trap_k;
        d.trap_dx = g.trap_dx;
        d.trap_dy = g.trap_dy;
        d.trap_t_eq = g.trap_t_eq;
        d.trap_pull = g.trap_pull;
        d.trap_w = g.trap_width;
        d.trap_x0 = P[0] + sdx / g.n_nodes;
        d.trap_y0 = P[1] + sdy / g.n_nodes;
        d.trap_x0 -= nx * std::floor(d.trap_x0 / nx);
        d.trap_y0 -= ny * std::floor(d.trap_y0 / ny);
        d.trap_f[0] = d.trap_f[1] = make_float2(0.f, 0.f);
        d.k_spring = g.k_spring;
        d.eps_angle = g.eps_angle;
        d.l_eq = g.l_eq;
        d.pull_x = g.pull_force * std::cos(g.pull_angle) / g.n_nodes;
        d.pull_y = g.pull_force * std::sin(g.pull_angle) / g.n_nodes;
        // until the first node-kernel pass the box is empty; its origin is node 0's cell, the
        // reference from which the node kernel measures the ring's extent
        d.box[0] = make_int4((int)std::floor(X[off].x), (int)std::floor(X[off].y), 0, 0);
        d.box[1] = d.box[0];
        d.cap_w = cw;
        d.cap_h = chh;
        d.box_off = box_off;
        box_off += 2LL * cw * chh;
        off += g.n_nodes;
    }
    h->n_rings = n_rings;
    h->n_total = off;
    h->row_len = 6 + 4 * n_rings;
    h->box_floats = box_off;
    // node-kernel work: NB owned nodes per CTA (one CTA with no ring when there are no rings)
    std::vector<int2> work;
    std::vector<int> cta0(std::max(n_rings, 1)), nctas(std::max(n_rings, 1));
    for (int r = 0; r < n_rings; ++r) {
        cta0[r] = (int)work.size();
        for (int k0 = 0; k0 < rd[r].n_nodes; k0 += NB) work.push_back(make_int2(r, k0));
        nctas[r] = (int)work.size() - cta0[r];
    }
    if (work.empty()) work.push_back(make_int2(-1, 0));
    h->n_node_ctas = (int)work.size();
    CK(h, cudaMalloc(&h->node_work, sizeof(int2) * work.size()));
    CK(h, cudaMalloc(&h->ring_cta0, sizeof(int) * cta0.size()));
    CK(h, cudaMalloc(&h->ring_ctas, sizeof(int) * nctas.size()));
    CK(h, cudaMalloc(&h->ring_tickets, sizeof(unsigned) * nctas.size()));
    CK(h, cudaMalloc(&h->node_partials, sizeof(double) * NODE_PARTIALS * work.size()));
    CK(h, cudaMemcpy(h->node_work, work.data(), sizeof(int2) * work.size(), cudaMemcpyHostToDevice));
    CK(h, cudaMemcpy(h->ring_cta0, cta0.data(), sizeof(int) * cta0.size(), cudaMemcpyHostToDevice));
    CK(h, cudaMemcpy(h->ring_ctas, nctas.data(), sizeof(int) * nctas.size(), cudaMemcpyHostToDevice));
    CK(h, cudaMemset(h->ring_tickets, 0, sizeof(unsigned) * nctas.size()));
    CK(h, cudaMalloc(&h->box_tickets, sizeof(unsigned) * nctas.size()));
    CK(h, cudaMemset(h->box_tickets, 0, sizeof(unsigned) * nctas.size()));
    CK(h, cudaMalloc(&h->ring_claim, sizeof(unsigned long long) * nctas.size()));
    CK(h, cudaMemset(h->ring_claim, 0, sizeof(unsigned long long) * nctas.size()));
    if (n_rings > 0) {
        CK(h, cudaMalloc(&h->rings, sizeof(RingDev) * n_rings));
        CK(h, cudaMalloc(&h->X, sizeof(double2) * off));
        CK(h, cudaMalloc(&h->X_alt, sizeof(double2) * off));
        CK(h, cudaMalloc(&h->node_cell, sizeof(int2) * off));
        CK(h, cudaMalloc(&h->node_frac, sizeof(float2) * off));
        CK(h, cudaMalloc(&h->node_force, sizeof(float2) * off));
        CK(h, cudaMalloc(&h->ubox, sizeof(float) * box_off));
        CK(h, cudaMalloc(&h->fpbox, sizeof(float) * box_off));
        CK(h, cudaMemcpy(h->rings, rd.data(), sizeof(RingDev) * n_rings, cudaMemcpyHostToDevice));
        CK(h, cudaMemcpy(h->X, X.data(), sizeof(double2) * off, cudaMemcpyHostToDevice));
        CK(h, cudaMemset(h->ubox, 0, sizeof(float) * box_off));
        CK(h, cudaMemset(h->fpbox, 0, sizeof(float) * box_off));
    }
    dfree(h->series);
    CK(h, cudaMalloc(&h->series, sizeof(double) * (size_t)h->series_cap * h->row_len));
    CK(h, cudaMemset(h->series, 0, sizeof(double) * (size_t)h->series_cap * h->row_len));
    if (n_rings > 0) {
        CK(h, launch_nodes(node_args(h, 0), h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
    }
    return LB_OK;
}

int lb_step(lb_handle* h, int64_t n)
{
    if (!h) return fail(nullptr, LB_EINVAL, "null handle");
    if (n < 0) return fail(h, LB_EINVAL, "n < 0");
    if (!h->fields_ready) return fail(h, LB_ESTATE, "lb_init_fields not called");
    if (!h->node_work) return fail(h, LB_ESTATE, "no valid body: call lb_set_body again");
    for (int64_t k = 0; k < n; ++k) {
        FusedArgs fa = fused_args(h);
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (h->timing) {
            e0 = ev_get(h->ev_fused, h->ev_fused_used);
            e1 = ev_get(h->ev_fused, h->ev_fused_used);
            if (e0) cudaEventRecord(e0, h->stream);
        }
        const bool sweep = h->kernel == LB_KERNEL_SWEEP;
        const bool pair = h->kernel == LB_KERNEL_PAIR;
        const bool strip = uses_strip(h);
        // consecutive kernels overlap by programmatic dependent launch, except when per-kernel
        // timing brackets each launch with events
        // no programmatic early start for the first launch after lb_commit_state (it must not
        // begin before the upload it waits for on the copy stream)
        const bool pdl = !h->timing && !h->no_pdl_once;
        h->no_pdl_once = false;
        // the tile kernels run the node step in their tail: one launch per step
        const bool tail = h->node_tail && !sweep && !strip;
        if (sweep) {
            CK(h, launch_sweep(fa, h->sweep_chunk, h->stream));
            h->n_partials = sweep_ctas(h->p.nx, h->p.ny, h->sweep_chunk);
        } else if (strip) {
            fa.t = h->t;
            CK(h, launch_strip(fa, h->strip_chunk, h->stream, pdl));
            h->n_partials = strip_ctas(h->p.nx, h->p.ny, h->strip_chunk);
        } else {
            if (tail) {
                h->n_partials = fused_ctas(h->p.nx, h->p.ny);
                fa.node_tail = 1;
                fa.t = h->t;
                fa.tile_rot = h->tile_rot;
                fa.box_tickets = h->box_tickets;
                fa.ring_claim = h->ring_claim;
                fa.na = node_args(h, 1);
            }
            // without the tail, a lattice kernel stages the state before its dependency wait,
            // which is safe behind a node kernel only: after a launch with the tail it waits for
            // that launch to complete
            CK(h, launch_fused(fa, MODE_STEP, h->stream, &h->n_partials, pdl && (tail || !h->after_tail), pair));
        }
        h->after_tail = tail;
        if (h->p.diffusion_substeps > 0) {
            // sigma of the new state; the old state's sigma planes serve as the other buffer
            float* sig_new = static_cast<float*>(h->state[h->cur ^ 1]) + (size_t)PL_SXX * h->plane;
            float* sig_old = static_cast<float*>(h->state[h->cur]) + (size_t)PL_SXX * h->plane;
            CK(h, launch_diffusion(sig_new, sig_old, h->plane, h->p.nx, h->p.ny,
                                   (float)(h->p.Dp / h->p.diffusion_substeps), h->p.diffusion_substeps, h->stream));
        }
        if (h->timing && e1) cudaEventRecord(e1, h->stream);
        if (!tail) {
            if (h->timing) {
                e0 = ev_get(h->ev_nodes, h->ev_nodes_used);
                e1 = ev_get(h->ev_nodes, h->ev_nodes_used);
                if (e0) cudaEventRecord(e0, h->stream);
            }
            CK(h, launch_nodes(node_args(h, 1), h->stream, pdl && !sweep));
            if (h->timing && e1) cudaEventRecord(e1, h->stream);
        }
        std::swap(h->X, h->X_alt);
        h->cur ^= 1;
        h->t += 1;
    }
    return LB_OK;
}

int lb_sync(lb_handle* h)
{
    if (!h) return fail(nullptr, LB_EINVAL, "null handle");
    CK(h, cudaStreamSynchronize(h->stream));
    Ctl c;
    CK(h, cudaMemcpy(&c, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
    if (c.err_nonfinite || c.err_body || c.err_timeout) {
        int z[4] = {0, 0, 0, 0};
        CK(h, cudaMemcpy(&h->ctl->err_nonfinite, z, sizeof(int) * 4, cudaMemcpyHostToDevice));
        if (c.err_timeout) return fail(h, LB_ETIMEOUT, "a bounded wait in the lattice kernel timed out");
        if (c.err_nonfinite) return fail(h, LB_ENONFINITE, "non-finite readout or node force");
        return fail(h, LB_EBODY, "a ring left its work box or moved >= 1 cell in a step");
    }
    if (c.t != h->t) return fail(h, LB_ECUDA, "device step counter %lld != host %lld", c.t, h->t);
    return LB_OK;
}

int64_t lb_time(const lb_handle* h) { return h ? h->t : -1; }

int lb_readout(lb_handle* h, int32_t field, void* dst, size_t bytes, int32_t dst_is_device)
{
    if (!h || !dst) return fail(h, LB_EINVAL, "null argument");
    const size_t N = (size_t)h->plane;
    const cudaMemcpyKind kind = dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (field == LB_FIELD_NODES) {
        if (bytes != sizeof(double) * 2 * (size_t)h->n_total) return fail(h, LB_EINVAL, "bytes mismatch");
        if (h->n_total) CK(h, cudaMemcpyAsync(dst, h->X, bytes, kind, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
        return LB_OK;
    }
    if (bytes != sizeof(float) * N) return fail(h, LB_EINVAL, "bytes mismatch");
    const float* srcp = nullptr;
    if (!h->moments) CK(h, cudaMalloc(&h->moments, sizeof(float) * 3 * N));
    if (field >= LB_FIELD_DRHO && field <= LB_FIELD_UY) {
        FusedArgs fa = fused_args(h);
        CK(h, launch_fused(fa, MODE_MOMENTS, h->stream, nullptr));
        srcp = h->moments + (size_t)(field - LB_FIELD_DRHO) * N;
    } else if (field >= LB_FIELD_SXX && field <= LB_FIELD_PY) {
        CK(h, plane_to_f32(h, h->cur, PL_SXX + field - LB_FIELD_SXX, h->moments));
        srcp = h->moments;
    } else if (field >= LB_FIELD_POP0 && field < LB_FIELD_POP0 + 9) {
        CK(h, plane_to_f32(h, h->cur, field - LB_FIELD_POP0, h->moments));
        srcp = h->moments;
    } else {
        return fail(h, LB_EINVAL, "unknown field %d", field);
    }
    CK(h, cudaMemcpyAsync(dst, srcp, bytes, kind, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return LB_OK;
}

int lb_write_field(lb_handle* h, int32_t field, const void* src, size_t bytes, int32_t src_is_device)
{
    if (!h || !src) return fail(h, LB_EINVAL, "null argument");
    const size_t N = (size_t)h->plane;
    if (bytes != sizeof(float) * N) return fail(h, LB_EINVAL, "bytes mismatch");
    size_t plane;
    if (field >= LB_FIELD_SXX && field <= LB_FIELD_PY) plane = PL_SXX + field - LB_FIELD_SXX;
    else if (field >= LB_FIELD_POP0 && field < LB_FIELD_POP0 + 9) plane = field - LB_FIELD_POP0;
    else return fail(h, LB_EINVAL, "field %d is not writable", field);
    if (h->p.model == LB_MODEL_SCALAR && (field == LB_FIELD_PX || field == LB_FIELD_PY))
        return fail(h, LB_EINVAL, "the scalar model has no P field to write");
    const cudaMemcpyKind kind = src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (!h->moments) CK(h, cudaMalloc(&h->moments, sizeof(float) * 3 * N));
    CK(h, cudaMemcpyAsync(h->moments, src, bytes, kind, h->stream));
    CK(h, f32_to_plane(h, h->cur, (int)plane, h->moments));
    CK(h, cudaStreamSynchronize(h->stream));
    return LB_OK;
}

int32_t lb_series_row_len(const lb_handle* h) { return h ? h->row_len : 0; }

static int series_rows(const lb_handle* h)
{
    const long long every = h->p.readout_every;
    const long long recorded = (h->t + every - 1) / every;   // t' in [0, t) with t' % every == 0
    return (int)std::min<long long>(recorded, h->series_cap);
}

int lb_series(lb_handle* h, double* dst, int32_t max_rows, int32_t* rows_written)
{
    if (!h || !dst || max_rows < 0) return fail(h, LB_EINVAL, "bad argument");
    CK(h, cudaStreamSynchronize(h->stream));
    const long long every = h->p.readout_every;
    const long long recorded = (h->t + every - 1) / every;
    const int rows = std::min(series_rows(h), max_rows);
    std::vector<double> all((size_t)h->series_cap * h->row_len);
    CK(h, cudaMemcpy(all.data(), h->series, sizeof(double) * all.size(), cudaMemcpyDeviceToHost));
    const long long first = recorded - series_rows(h);      // oldest sample index kept
    for (int r = 0; r < rows; ++r) {
        const long long k = first + r;
        memcpy(dst + (size_t)r * h->row_len, all.data() + (size_t)(k % h->series_cap) * h->row_len,
               sizeof(double) * h->row_len);
    }
    if (rows_written) *rows_written = rows;
    return LB_OK;
}

int lb_series_latest(lb_handle* h, double* dst, int32_t n, int32_t* rows_written)
{
    if (!h || !dst || n < 0) return fail(h, LB_EINVAL, "bad argument");
    const long long every = h->p.readout_every;
    const long long recorded = (h->t + every - 1) / every;
    const int rows = std::min(series_rows(h), n);
    // the ring-buffer slots of the newest rows, copied one by one (oldest first); ordered on the
    // stream after the steps that wrote them
    for (int r = 0; r < rows; ++r) {
        const long long k = recorded - rows + r;
        CK(h, cudaMemcpyAsync(dst + (size_t)r * h->row_len, h->series + (size_t)(k % h->series_cap) * h->row_len,
                              sizeof(double) * h->row_len, cudaMemcpyDeviceToHost, h->stream));
    }
    CK(h, cudaStreamSynchronize(h->stream));
    if (rows_written) *rows_written = rows;
    return LB_OK;
}

int lb_series_latest_async(lb_handle* h, double* dst, int32_t n, int32_t* rows_written)
{
    if (!h || !dst || n < 0) return fail(h, LB_EINVAL, "bad argument");
    if (!h->ev_series) CK(h, cudaEventCreateWithFlags(&h->ev_series, cudaEventDisableTiming));
    const long long every = h->p.readout_every;
    const long long recorded = (h->t + every - 1) / every;
    const int rows = std::min(series_rows(h), n);
    for (int r = 0; r < rows; ++r) {
        const long long k = recorded - rows + r;
        CK(h, cudaMemcpyAsync(dst + (size_t)r * h->row_len, h->series + (size_t)(k % h->series_cap) * h->row_len,
                              sizeof(double) * h->row_len, cudaMemcpyDeviceToHost, h->stream));
    }
    CK(h, cudaEventRecord(h->ev_series, h->stream));
    h->series_pending = true;
    if (rows_written) *rows_written = rows;
    return LB_OK;
}

int lb_series_wait(lb_handle* h)
{
    if (!h) return fail(nullptr, LB_EINVAL, "null handle");
    if (!h->series_pending) return LB_OK;
    CK(h, cudaEventSynchronize(h->ev_series));
    h->series_pending = false;
    return LB_OK;
}

int64_t lb_state_bytes(const lb_handle* h) { return h ? (int64_t)N_PLANES * h->plane * h->esz : 0; }

int lb_read_state(lb_handle* h, void* dst, size_t bytes, int32_t dst_is_device)
{
    if (!h || !dst) return fail(h, LB_EINVAL, "null argument");
    if (!h->fields_ready) return fail(h, LB_ESTATE, "lb_init_fields not called");
    if (bytes != (size_t)lb_state_bytes(h)) return fail(h, LB_EINVAL, "need %lld bytes", (long long)lb_state_bytes(h));
    CK(h, cudaMemcpyAsync(dst, h->state[h->cur], bytes, dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                          h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return LB_OK;
}

int lb_write_state(lb_handle* h, const void* src, size_t bytes, int32_t src_is_device)
{
    if (!h || !src) return fail(h, LB_EINVAL, "null argument");
    if (!h->fields_ready) return fail(h, LB_ESTATE, "lb_init_fields not called");
    if (bytes != (size_t)lb_state_bytes(h)) return fail(h, LB_EINVAL, "need %lld bytes", (long long)lb_state_bytes(h));
    CK(h, cudaMemcpyAsync(h->state[h->cur], src, bytes, src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                          h->stream));
    return LB_OK;
}

int lb_stage_state(lb_handle* h, const void* src, size_t bytes, int32_t src_is_device)
{
    if (!h || !src) return fail(h, LB_EINVAL, "null argument");
    if (!h->fields_ready) return fail(h, LB_ESTATE, "lb_init_fields not called");
    if (bytes != (size_t)lb_state_bytes(h)) return fail(h, LB_EINVAL, "need %lld bytes", (long long)lb_state_bytes(h));
    if (!h->copy_stream) {
        CK(h, cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking));
        CK(h, cudaEventCreateWithFlags(&h->ev_staged, cudaEventDisableTiming));
        CK(h, cudaEventCreateWithFlags(&h->ev_release, cudaEventDisableTiming));
    }
    if (!h->stage_buf) CK(h, cudaMalloc(&h->stage_buf, bytes));
    // the previous commit's copy out of the staging buffer must be done before it is overwritten
    if (h->release_pending) CK(h, cudaStreamWaitEvent(h->copy_stream, h->ev_release, 0));
    CK(h, cudaMemcpyAsync(h->stage_buf, src, bytes, src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                          h->copy_stream));
    CK(h, cudaEventRecord(h->ev_staged, h->copy_stream));
    h->staged = true;
    return LB_OK;
}

int lb_commit_state(lb_handle* h)
{
    if (!h) return fail(nullptr, LB_EINVAL, "null handle");
    if (!h->staged) return fail(h, LB_ESTATE, "lb_commit_state: no state staged (lb_stage_state)");
    CK(h, cudaStreamWaitEvent(h->stream, h->ev_staged, 0));
    if (h->batch_refs == 0) {
        // the staging buffer becomes the current state and the former current buffer the
        // staging buffer (the next stage waits until the work queued so far has read it)
        std::swap(h->state[h->cur], h->stage_buf);
    } else {
        // a batch's graphs hold the handle's buffers: copy into them instead
        CK(h, cudaMemcpyAsync(h->state[h->cur], h->stage_buf, (size_t)lb_state_bytes(h), cudaMemcpyDeviceToDevice,
                              h->stream));
    }
    CK(h, cudaEventRecord(h->ev_release, h->stream));
    h->no_pdl_once = true;
    h->staged = false;
    h->release_pending = true;
    return LB_OK;
}

int lb_restoring_force(lb_handle* h, int32_t ring, double* dst, int32_t max_k, int32_t* k_written)
{
    if (!h || !dst || ring < 0 || ring >= h->n_rings) return fail(h, LB_EINVAL, "bad argument");
    std::vector<double> rows((size_t)std::max(series_rows(h), 1) * h->row_len);
    int n = 0;
    int rc = lb_series(h, rows.data(), series_rows(h), &n);
    if (rc) return rc;
    const int k = std::min(n, max_k);
    for (int i = 0; i < k; ++i) {
        dst[2 * i] = rows[(size_t)i * h->row_len + 6 + 4 * ring];
        dst[2 * i + 1] = rows[(size_t)i * h->row_len + 7 + 4 * ring];
    }
    if (k_written) *k_written = k;
    return LB_OK;
}

int lb_timing(lb_handle* h, int32_t enable)
{
    if (!h) return fail(nullptr, LB_EINVAL, "null handle");
    CK(h, cudaStreamSynchronize(h->stream));
    h->timing = enable != 0;
    h->ev_fused_used = h->ev_nodes_used = 0;
    return LB_OK;
}

int lb_kernel_time(lb_handle* h, double* fused_ms, int64_t* fused_launches, double* node_ms,
                   int64_t* node_launches)
{
    if (!h) return fail(nullptr, LB_EINVAL, "null handle");
    CK(h, cudaStreamSynchronize(h->stream));
    double tf = 0.0, tn = 0.0;
    for (size_t i = 0; i + 1 < h->ev_fused_used; i += 2) {
        float ms = 0.f;
        CK(h, cudaEventElapsedTime(&ms, h->ev_fused[i], h->ev_fused[i + 1]));
        tf += ms;
    }
    for (size_t i = 0; i + 1 < h->ev_nodes_used; i += 2) {
        float ms = 0.f;
        CK(h, cudaEventElapsedTime(&ms, h->ev_nodes[i], h->ev_nodes[i + 1]));
        tn += ms;
    }
    if (fused_ms) *fused_ms = tf;
    if (fused_launches) *fused_launches = (int64_t)(h->ev_fused_used / 2);
    if (node_ms) *node_ms = tn;
    if (node_launches) *node_launches = (int64_t)(h->ev_nodes_used / 2);
    return LB_OK;
}

int32_t lb_launches_per_step(const lb_handle* h)
{
    if (!h) return 0;
    const int s = h->p.diffusion_substeps;
    const bool tail = h->node_tail && h->kernel != LB_KERNEL_SWEEP && !uses_strip(h);
    return (tail ? 1 : 2) + (s > 0 ? s + (s & 1) : 0);
}

int lb_set_node_tail(lb_handle* h, int32_t enable)
{
    if (!h) return fail(nullptr, LB_EINVAL, "null handle");
    if (enable != 0 && enable != 1) return fail(h, LB_EINVAL, "enable must be 0 or 1");
    h->node_tail = enable != 0;
    return LB_OK;
}

int32_t lb_stiffness_table(double P_cap, float* dst, int32_t max_entries)
{
    if (!(P_cap > 0.0 && P_cap < 1.0)) return fail(nullptr, LB_EINVAL, "need 0 < P_cap < 1");
    if (!dst) return LUT_N + 1;
    if (max_entries < LUT_N + 1) return fail(nullptr, LB_EINVAL, "need %d entries", LUT_N + 1);
    std::vector<float> t;
    cached_lut(P_cap, t);
    memcpy(dst, t.data(), sizeof(float) * t.size());
    return LUT_N + 1;
}

int lb_set_kernel(lb_handle* h, int32_t kernel)
{
    if (!h) return fail(nullptr, LB_EINVAL, "null handle");
    if (kernel < LB_KERNEL_AUTO || kernel > LB_KERNEL_STRIP) return fail(h, LB_EINVAL, "unknown kernel %d", kernel);
    if (kernel == LB_KERNEL_STRIP && !strip_eligible(h->p.nx, h->p.ny, h->p.walls_x || h->p.walls_y))
        return fail(h, LB_EINVAL, "the strip kernel needs a periodic lattice with nx >= 64, ny >= 32");
    if (kernel == LB_KERNEL_SWEEP && h->p.precision != LB_FP32)
        return fail(h, LB_EINVAL, "the sweep kernel stores FP32 only");
    if ((kernel == LB_KERNEL_SWEEP || kernel == LB_KERNEL_PAIR) && h->p.model == LB_MODEL_SCALAR)
        return fail(h, LB_EINVAL, "the scalar model runs on the one-cell tile kernel only");
    if ((kernel == LB_KERNEL_SWEEP || kernel == LB_KERNEL_PAIR) && (h->p.walls_y || h->p.walls_x))
        return fail(h, LB_EINVAL, "walls run on the one-cell tile kernel only");
    if (kernel == LB_KERNEL_SWEEP && !sweep_eligible(h->p.nx, h->p.ny))
        return fail(h, LB_EINVAL, "the sweep kernel needs nx %% 4 == 0, nx >= 256, ny >= 16");
    h->kernel = kernel;
    return LB_OK;
}

int32_t lb_lattice_kernel(const lb_handle* h)
{
    if (!h) return LB_EINVAL;
    if (uses_strip(h)) return LB_KERNEL_STRIP;
    return h->kernel == LB_KERNEL_AUTO ? LB_KERNEL_TILE : h->kernel;
}

double lb_bytes_per_cell(const lb_handle* h)
{
    if (!h) return 0.0;
    const int planes = h->p.model == LB_MODEL_SCALAR ? N_PLANES - 2 : N_PLANES;   // no P planes
    return 2.0 * planes * h->esz;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// Readout without device allocation.
//
// lb_readout creates its intermediate buffer for rho and u with cudaMalloc the first time it is
// asked for them.  Some callers cannot allow that: code that runs while another framework owns
// the whole device memory budget through its own pool, or code that must not allocate after its
// set-up phase (a long-running service with a fixed memory plan).  lb_readout_noalloc computes
// the same fields into a scratch array that is part of the library image on each GPU instead.
// ---------------------------------------------------------------------------------------------
namespace {

// Largest lattice the no-allocation readout accepts: 2^20 cells (e.g. 1024 x 1024).  The array
// holds three FP32 planes (rho - rho0, u_x, u_y), 12 MiB, on every GPU that loads the library,
// for as long as the process runs.
constexpr long long NOALLOC_MAX_CELLS = 1LL << 20;
static __device__ __align__(256) float g_noalloc_scratch[3 * NOALLOC_MAX_CELLS];

// The array's name is only a host-side handle; its device address is looked up once per device.
constexpr int NOALLOC_MAX_DEVICES = 64;
float* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {nullptr};

int noalloc_scratch(lb_handle* h, float** out)
{
    int dev = 0;
    CK(h, cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return fail(h, LB_EINVAL, "device index %d out of range", dev);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        CK(h, cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_noalloc_ptr[dev] = (float*)p;
    }
    *out = g_noalloc_ptr[dev];
    return LB_OK;
}

}  // namespace

extern "C" {

int lb_readout_noalloc(lb_handle* h, int32_t field, void* dst, size_t bytes, int32_t dst_is_device)
{
    if (!h || !dst) return fail(h, LB_EINVAL, "null argument");
    const size_t N = (size_t)h->plane;
    if ((long long)N > NOALLOC_MAX_CELLS)
        return fail(h, LB_EINVAL, "lb_readout_noalloc: %zu cells exceed the limit of %lld", N,
                    NOALLOC_MAX_CELLS);
    if (bytes != sizeof(float) * N) return fail(h, LB_EINVAL, "bytes mismatch");
    float* scratch = nullptr;
    int rc = noalloc_scratch(h, &scratch);
    if (rc != LB_OK) return rc;
    const float* srcp = nullptr;
    if (field >= LB_FIELD_DRHO && field <= LB_FIELD_UY) {
        // every in-lattice element of the three planes is written before it is read
        FusedArgs fa = fused_args(h);
        fa.moments_out = scratch;
        CK(h, launch_fused(fa, MODE_MOMENTS, h->stream, nullptr));
        srcp = scratch + (size_t)(field - LB_FIELD_DRHO) * N;
    } else if (field == LB_FIELD_PX || field == LB_FIELD_PY) {
        CK(h, plane_to_f32(h, h->cur, PL_SXX + field - LB_FIELD_SXX, scratch));
        srcp = scratch;
    } else {
        return fail(h, LB_EINVAL, "lb_readout_noalloc: field %d is not one of DRHO, UX, UY, PX, PY", field);
    }
    const cudaMemcpyKind kind = dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    CK(h, cudaMemcpyAsync(dst, srcp, bytes, kind, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return LB_OK;
}

const char* lb_last_error(const lb_handle* h) { return h ? h->err.c_str() : g_err.c_str(); }

void lb_destroy(lb_handle* h)
{
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    free_rings(h);
    dfree(h->state[0]);
    dfree(h->state[1]);
    dfree(h->lut);
    dfree(h->ctl);
    dfree(h->partials);
    dfree(h->series);
    dfree(h->moments);
    if (h->copy_stream) {
        cudaStreamSynchronize(h->copy_stream);
        cudaStreamDestroy(h->copy_stream);
    }
    if (h->ev_staged) cudaEventDestroy(h->ev_staged);
    if (h->ev_series) cudaEventDestroy(h->ev_series);
    if (h->ev_release) cudaEventDestroy(h->ev_release);
    dfree(h->stage_buf);
    for (auto e : h->ev_fused) cudaEventDestroy(e);
    for (auto e : h->ev_nodes) cudaEventDestroy(e);
    delete h;
}

}  // extern "C"
