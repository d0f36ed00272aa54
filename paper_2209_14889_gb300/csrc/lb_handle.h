// lb_handle.h -- the solver handle behind the C ABI (host side; shared by lb_api.cu and
// lb_batch.cu).
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/lb.h"
#include "lb_internal.h"

using vlb::Ctl;
using vlb::Phys;
using vlb::RingDev;

struct lb_handle {
    lb_params p;
    cudaStream_t stream = nullptr;
    Phys ph;
    double eta_p = 0.0;
    long long plane = 0;
    void* state[2] = {nullptr, nullptr};    // N_PLANES planes each (FP32, or 2-byte in LB_FP16_BF16)
    int esz = 4;                            // bytes per stored value
    int cur = 0;
    float2* lut = nullptr;
    Ctl* ctl = nullptr;
    double* partials = nullptr;
    int partial_cap = 0;                    // capacity of partials (tiles of the largest launch)
    int n_partials = 0;                     // partial sums written by the last lattice launch
    int kernel = 0;                         // LB_KERNEL_AUTO / TILE / SWEEP / PAIR / STRIP
    int sweep_chunk = 0;
    int strip_chunk = 0;                    // rows per warp of the strip kernel
    int n_sm = 152;                         // multiprocessors of the handle's device
    double* series = nullptr;
    int series_cap = 0;
    int row_len = 6;
    float* moments = nullptr;               // 3 planes, allocated on first use
    // rings
    int n_rings = 0, n_total = 0;
    RingDev* rings = nullptr;
    double2* X = nullptr;                   // node positions of the current step
    double2* X_alt = nullptr;               // the other position buffer: an advancing node launch
                                            // reads X and writes X_alt, then the two swap
    int2* node_cell = nullptr;
    float2* node_frac = nullptr;
    float2* node_force = nullptr;
    float* ubox = nullptr;
    float* fpbox = nullptr;
    int n_node_ctas = 1;
    int2* node_work = nullptr;
    int* ring_cta0 = nullptr;
    int* ring_ctas = nullptr;
    unsigned* ring_tickets = nullptr;
    unsigned* box_tickets = nullptr;        // per ring: tile arrivals of the node tail
    unsigned long long* ring_claim = nullptr;   // per ring: open node blocks of the node tail
    bool node_tail = true;                  // node step in the lattice kernel's tail (tile kernels)
    bool after_tail = false;                // the last lattice launch ran the node tail
    int tile_rot = 0;                       // first tile row of the tail launches
    double* node_partials = nullptr;
    long long box_floats = 0;
    bool fields_ready = false;
    long long t = 0;
    // lb_stage_state / lb_commit_state: a staged copy of a whole stored state, uploaded on a copy
    // stream while the handle's stream computes (allocated on first use)
    void* stage_buf = nullptr;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_staged = nullptr;        // the upload into stage_buf is complete
    cudaEvent_t ev_release = nullptr;       // the handle's stream has read stage_buf
    bool staged = false, release_pending = false;
    int batch_refs = 0;                     // live batches holding this handle's buffers
    bool no_pdl_once = false;               // the next lattice launch starts without PDL
    cudaEvent_t ev_series = nullptr;        // lb_series_latest_async: its copies are done
    bool series_pending = false;
    // timing
    bool timing = false;
    std::vector<cudaEvent_t> ev_fused, ev_nodes;
    size_t ev_fused_used = 0, ev_nodes_used = 0;
    std::string err;
};

namespace vlb {
// argument blocks of the two kernels of a step for the handle's current buffers (lb_api.cu)
FusedArgs handle_fused_args(lb_handle* h);
NodeArgs handle_node_args(lb_handle* h, int advance);
}  // namespace vlb
