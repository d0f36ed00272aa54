// lb_ckpt.cu -- lb_save / lb_load (include/lb.h): a raw snapshot of a handle's state.
//
// The snapshot lists every device buffer that a step carries over to the next one, with the size
// the handle allocated for it, plus the host-side step counter, current buffer index and launch
// flags.  Buffers that only describe the ring layout (node work lists, CTA offsets), the C~ table
// and scratch arrays are not stored: a handle with equal parameters and the same ring layout
// already holds them.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "lb_handle.h"

namespace {

constexpr char kMagic[8] = {'V', 'L', 'B', 'C', 'K', 'P', 'T', '1'};
constexpr uint32_t kVersion = 1;

// Everything that must agree between the saving and the loading handle, then the host state.
struct Header {
    char magic[8];
    uint32_t version;
    uint32_t header_bytes;
    lb_params p;
    int64_t plane, box_floats;
    int32_t esz, partial_cap, series_cap, row_len;
    int32_t n_rings, n_total, n_node_ctas, n_bufs;
    int64_t payload_bytes;
    // host state
    int64_t t;
    int32_t cur, after_tail, tile_rot, n_partials;
};

struct Buf {
    void* ptr;
    size_t bytes;
};

// The buffers of the snapshot, in file order; a null pointer stands for a buffer the handle does
// not have (no rings yet), and is stored as zero bytes.
std::vector<Buf> snapshot_bufs(lb_handle* h)
{
    const size_t state_bytes = (size_t)h->esz * vlb::N_PLANES * (size_t)h->plane;
    const size_t nr = (size_t)(h->n_rings > 0 ? h->n_rings : 1);     // ticket arrays hold >= 1
    const size_t nt = (size_t)h->n_total;
    auto B = [](void* p, size_t n) { return Buf{p, p ? n : 0}; };
    return {
        B(h->state[0], state_bytes),
        B(h->state[1], state_bytes),
        B(h->ctl, sizeof(vlb::Ctl)),
        B(h->partials, sizeof(double) * 5 * (size_t)h->partial_cap),
        B(h->series, sizeof(double) * (size_t)h->series_cap * (size_t)h->row_len),
        B(h->rings, sizeof(vlb::RingDev) * (size_t)h->n_rings),
        B(h->X, sizeof(double2) * nt),
        B(h->X_alt, sizeof(double2) * nt),
        B(h->node_cell, sizeof(int2) * nt),
        B(h->node_frac, sizeof(float2) * nt),
        B(h->node_force, sizeof(float2) * nt),
        B(h->ubox, sizeof(float) * (size_t)h->box_floats),
        B(h->fpbox, sizeof(float) * (size_t)h->box_floats),
        B(h->ring_tickets, sizeof(unsigned) * nr),
        B(h->box_tickets, sizeof(unsigned) * nr),
        B(h->ring_claim, sizeof(unsigned long long) * nr),
        B(h->node_partials, sizeof(double) * vlb::NODE_PARTIALS * (size_t)h->n_node_ctas),
    };
}

Header make_header(lb_handle* h, const std::vector<Buf>& bufs)
{
    Header hd;
    memset(&hd, 0, sizeof hd);
    memcpy(hd.magic, kMagic, sizeof kMagic);
    hd.version = kVersion;
    hd.header_bytes = sizeof(Header);
    hd.p = h->p;
    hd.plane = h->plane;
    hd.box_floats = h->box_floats;
    hd.esz = h->esz;
    hd.partial_cap = h->partial_cap;
    hd.series_cap = h->series_cap;
    hd.row_len = h->row_len;
    hd.n_rings = h->n_rings;
    hd.n_total = h->n_total;
    hd.n_node_ctas = h->n_node_ctas;
    hd.n_bufs = (int32_t)bufs.size();
    hd.payload_bytes = 0;
    for (const Buf& b : bufs) hd.payload_bytes += (int64_t)b.bytes;
    hd.t = h->t;
    hd.cur = h->cur;
    hd.after_tail = h->after_tail ? 1 : 0;
    hd.tile_rot = h->tile_rot;
    hd.n_partials = h->n_partials;
    return hd;
}

// lb_params compared field by field (padding bytes may differ between callers).
bool same_params(const lb_params& a, const lb_params& b)
{
    return a.nx == b.nx && a.ny == b.ny && a.tau == b.tau && a.rho0 == b.rho0 && a.K1111 == b.K1111 &&
           a.K1122 == b.K1122 && a.K2222 == b.K2222 && a.K1212 == b.K1212 && a.eta_p == b.eta_p &&
           a.lambda_steps == b.lambda_steps && a.Dp == b.Dp && a.alpha == b.alpha && a.beta == b.beta &&
           a.xi == b.xi && a.Gamma == b.Gamma && a.kappa == b.kappa && a.P_cap == b.P_cap &&
           a.director_angle == b.director_angle && a.ericksen == b.ericksen && a.precision == b.precision &&
           a.readout_every == b.readout_every && a.max_samples == b.max_samples &&
           a.diffusion_substeps == b.diffusion_substeps && a.model == b.model && a.walls_y == b.walls_y &&
           a.walls_x == b.walls_x;
}

// The layout part of two headers (everything but the host state) agrees.
bool same_layout(const Header& a, const Header& b)
{
    return same_params(a.p, b.p) && a.plane == b.plane && a.box_floats == b.box_floats && a.esz == b.esz &&
           a.partial_cap == b.partial_cap && a.series_cap == b.series_cap && a.row_len == b.row_len &&
           a.n_rings == b.n_rings && a.n_total == b.n_total && a.n_node_ctas == b.n_node_ctas &&
           a.n_bufs == b.n_bufs && a.payload_bytes == b.payload_bytes;
}

int set_err(lb_handle* h, int code, const std::string& msg)
{
    h->err = msg;
    return code;
}

int cuda_err(lb_handle* h, cudaError_t e, const char* what)
{
    return set_err(h, e == cudaErrorMemoryAllocation ? LB_ENOMEM : LB_ECUDA,
                   std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace

extern "C" {

int lb_save(lb_handle* h, const char* path)
{
    if (!h) return LB_EINVAL;
    if (!path) return set_err(h, LB_EINVAL, "lb_save: null path");
    if (!h->fields_ready) return set_err(h, LB_ESTATE, "lb_save: lb_init_fields not called");
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_err(h, e, "lb_save: cudaStreamSynchronize");
    const std::vector<Buf> bufs = snapshot_bufs(h);
    const Header hd = make_header(h, bufs);
    std::vector<char> host((size_t)hd.payload_bytes);
    size_t off = 0;
    for (const Buf& b : bufs) {
        if (b.bytes) {
            e = cudaMemcpyAsync(host.data() + off, b.ptr, b.bytes, cudaMemcpyDeviceToHost, h->stream);
            if (e != cudaSuccess) return cuda_err(h, e, "lb_save: copy to host");
        }
        off += b.bytes;
    }
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_err(h, e, "lb_save: cudaStreamSynchronize");
    FILE* f = fopen(path, "wb");
    if (!f) return set_err(h, LB_EINVAL, std::string("lb_save: cannot open ") + path);
    const bool ok = fwrite(&hd, sizeof hd, 1, f) == 1 &&
                    (host.empty() || fwrite(host.data(), host.size(), 1, f) == 1);
    const bool closed = fclose(f) == 0;
    if (!ok || !closed) return set_err(h, LB_EINVAL, std::string("lb_save: cannot write ") + path);
    return LB_OK;
}

int lb_load(lb_handle* h, const char* path)
{
    if (!h) return LB_EINVAL;
    if (!path) return set_err(h, LB_EINVAL, "lb_load: null path");
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_err(h, e, "lb_load: cudaStreamSynchronize");
    const std::vector<Buf> bufs = snapshot_bufs(h);
    const Header mine = make_header(h, bufs);
    // read and check the whole file before touching the handle
    FILE* f = fopen(path, "rb");
    if (!f) return set_err(h, LB_EINVAL, std::string("lb_load: cannot open ") + path);
    Header hd;
    memset(&hd, 0, sizeof hd);
    bool ok = fread(&hd, sizeof hd, 1, f) == 1;
    if (ok && (memcmp(hd.magic, kMagic, sizeof kMagic) != 0 || hd.version != kVersion ||
               hd.header_bytes != sizeof(Header))) {
        fclose(f);
        return set_err(h, LB_EINVAL, "lb_load: not a checkpoint of this library version");
    }
    if (ok && !same_layout(hd, mine)) {
        fclose(f);
        return set_err(h, LB_EINVAL, "lb_load: the checkpoint's parameters or ring layout differ from the handle's");
    }
    std::vector<char> host;
    if (ok) {
        host.resize((size_t)hd.payload_bytes);
        ok = host.empty() || fread(host.data(), host.size(), 1, f) == 1;
        char extra;
        ok = ok && fread(&extra, 1, 1, f) == 0;                    // nothing after the payload
    }
    fclose(f);
    if (!ok) return set_err(h, LB_EINVAL, std::string("lb_load: truncated or malformed file ") + path);
    if (hd.cur != 0 && hd.cur != 1) return set_err(h, LB_EINVAL, "lb_load: malformed file (buffer index)");
    if (h->n_rings > 0) {
        // the ring records must describe this handle's layout (node ranges, box capacities and
        // offsets), not only the same totals
        size_t roff = 0;
        for (const Buf& b : bufs) {
            if (b.ptr == h->rings) break;
            roff += b.bytes;
        }
        std::vector<vlb::RingDev> theirs(h->n_rings), ours(h->n_rings);
        memcpy(theirs.data(), host.data() + roff, sizeof(vlb::RingDev) * theirs.size());
        e = cudaMemcpyAsync(ours.data(), h->rings, sizeof(vlb::RingDev) * ours.size(), cudaMemcpyDeviceToHost,
                            h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return cuda_err(h, e, "lb_load: ring records");
        for (size_t r = 0; r < ours.size(); ++r) {
            const vlb::RingDev &a = theirs[r], &b = ours[r];
            if (a.n_nodes != b.n_nodes || a.node_off != b.node_off || a.cap_w != b.cap_w ||
                a.cap_h != b.cap_h || a.box_off != b.box_off)
                return set_err(h, LB_EINVAL, "lb_load: the checkpoint's ring layout differs from the handle's");
            // the ring's constant physics (spring, angle term, rest length, pull, trap protocol)
            // must be the handle's: a load restores the state of a run, not its parameters.  The
            // trap's origin and force slots are state and come from the file.
            if (a.k_spring != b.k_spring || a.eps_angle != b.eps_angle || a.l_eq != b.l_eq ||
                a.pull_x != b.pull_x || a.pull_y != b.pull_y || a.trap_k != b.trap_k ||
                a.trap_dx != b.trap_dx || a.trap_dy != b.trap_dy || a.trap_t_eq != b.trap_t_eq ||
                a.trap_pull != b.trap_pull || a.trap_w != b.trap_w)
                return set_err(h, LB_EINVAL, "lb_load: ring " + std::to_string(r) + "'s parameters differ from the handle's");
        }
    }
    size_t off = 0;
    for (const Buf& b : bufs) {
        if (b.bytes) {
            e = cudaMemcpyAsync(b.ptr, host.data() + off, b.bytes, cudaMemcpyHostToDevice, h->stream);
            if (e != cudaSuccess) return cuda_err(h, e, "lb_load: copy to device (handle state undefined)");
        }
        off += b.bytes;
    }
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_err(h, e, "lb_load: cudaStreamSynchronize (handle state undefined)");
    h->t = hd.t;
    h->cur = hd.cur;
    h->after_tail = hd.after_tail != 0;
    h->tile_rot = hd.tile_rot;
    h->n_partials = hd.n_partials;
    h->fields_ready = true;
    return LB_OK;
}

}  // extern "C"
