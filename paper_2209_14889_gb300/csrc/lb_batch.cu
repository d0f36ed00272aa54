// lb_batch.cu -- batched sweeps: many independent lattices of uneven sizes advanced together,
// a chunk of steps per captured CUDA graph.
//
// Default (phase launches): each step is one launch per phase and tile-shape group -- all
// instances' lattice tiles (k_batch_tiles, the tile kernel's occupancy of three CTAs per SM),
// their diffusion sub-steps, then their node blocks -- in stream order, so no kernel waits on
// another inside a launch.  Alternatively (lb_batch_set_persistent) one persistent cooperative
// kernel per group runs the whole chunk, each step having three phases separated by a grid
// barrier:
//   lattice  the fused step of every tile of every instance (tile shape per instance, chosen by
//            the autotuner among 32x16, 32x8, 64x8, 16x16), the tile code of lb_tile.cuh;
//   sigma    diffusion sub-steps of the instances whose D_p exceeds the Heun bound;
//   nodes    the node blocks of every ring of every instance (lb_node.cuh).
// Work items are assigned to CTAs round-robin, so the schedule and every result are the same
// from run to run.  The barrier spins with an iteration limit and reports LB_ETIMEOUT.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "lb_diffuse.cuh"
#include "lb_handle.h"
#include "lb_node.cuh"
#include "lb_strip.cuh"
#include "lb_tile.cuh"

namespace vlb {
namespace {

constexpr int BT = 256;     // threads per CTA
// tile shapes 0..3 (32x16, 32x8, 64x8, 16x16 cells per CTA), and shape 4: the warp-strip kernel
// (phase launches only; a CTA = SWARPS strips of SOWN columns x STRIP_H rows)
constexpr int N_SHAPES = 5;
constexpr int N_TILE_SHAPES = 4;
constexpr int SHAPE_STRIP = 4;
constexpr int STRIP_H = 64;
__host__ __device__ constexpr int shape_tx(int s) { return s == 0 ? 32 : (s == 1 ? 32 : (s == 2 ? 64 : 16)); }
__host__ __device__ constexpr int shape_ty(int s) { return s == 0 ? 16 : (s == 1 ? 8 : (s == 2 ? 8 : 16)); }

constexpr size_t cmaxz(size_t a, size_t b) { return a > b ? a : b; }
// dynamic shared memory of the kernel of one tile shape
template <int TX, int TY>
constexpr size_t batch_smem() { return cmaxz(tile::TileGeo<TX, TY>::SMEM_BYTES, sizeof(float) * dif::SMEM); }

struct BatchInst {
    FusedArgs fa[2];            // lattice step from buffer p to buffer p^1, p = 0, 1
    NodeArgs na;
    float* sig[2];              // sigma planes of buffer 0 and 1
    double2* xb[2];             // node positions read in a step whose lattice source is buffer p
    int shape, tiles_x, tiles_y;
    int dsub;                   // diffusion sub-steps (0: none)
    float dsub_D;               // D_p / dsub
    int dif_tx, dif_ty;
};

struct BatchArgs {
    const BatchInst* inst;
    int n_inst;
    const int* tile_begin;      // prefix sums of lattice tiles over instances (n_inst + 1)
    const int* node_begin;      // prefix sums of node blocks
    const int* dif_begin;       // prefix sums of diffusion tiles (instances with dsub > 0)
    int max_dsub;
    int* cur;                   // buffer parity of the current state (device)
    unsigned* bar;              // [0] arrivals, [1] generation
    int* err;                   // barrier timeout flag
    unsigned extra_arrivals;    // 0; > 0 only to exercise the timeout path
    unsigned long long wait_ns; // limit of one barrier wait
};

__device__ __forceinline__ int find_inst(const int* begin, int n, int item)
{
    int lo = 0, hi = n;          // begin[lo] <= item < begin[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (begin[mid] <= item) lo = mid; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier of a cooperative launch (all CTAs are co-resident).  The wait gives up after
// B.wait_ns (or 2^26 polls), sets the error flag and returns false; the caller then stops.
__device__ bool grid_sync(const BatchArgs& B)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* gen = B.bar + 1;
        const unsigned g = *gen;
        __threadfence();
        int ok = 1;
        if (atomicAdd(B.bar, 1u) == gridDim.x - 1 + B.extra_arrivals) {
            B.bar[0] = 0u;
            __threadfence();
            atomicAdd(B.bar + 1, 1u);
        } else {
            const unsigned long long t0 = global_ns();
            unsigned it = 0;
            while (*gen == g) {
                if (++it > (1u << 26) || global_ns() - t0 > B.wait_ns) {
                    atomicExch(B.err, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// One kernel per tile shape: the instances of a batch are grouped by their shape and each group
// runs its own persistent launch (one tile body per kernel keeps within the register budget of
// two 256-thread CTAs per SM; the instances are independent, so the groups need no common
// barrier).
template <int TX, int TY, bool SCALAR>
__global__ void __launch_bounds__(BT, 2) k_batch(const BatchArgs B, int nsteps)
{
    extern __shared__ __align__(16) float sm[];
    const int cur0 = *B.cur;
    const int n_tiles = __ldg(B.tile_begin + B.n_inst), n_nodes = __ldg(B.node_begin + B.n_inst);
    const int n_dif = __ldg(B.dif_begin + B.n_inst);
    bool ok = true;
    for (int s = 0; s < nsteps && ok; ++s) {
        const int par = (cur0 + s) & 1;
        for (int item = blockIdx.x; item < n_tiles; item += gridDim.x) {
            const int i = find_inst(B.tile_begin, B.n_inst, item);
            const BatchInst& I = B.inst[i];
            const int local = item - __ldg(B.tile_begin + i);
            const int by = local / I.tiles_x, bx = local - by * I.tiles_x;
            // the tile step of lb_step; coherent loads: the state was written by the previous step
            // of this launch
            tile::tile_step<MODE_STEP, cell::PREC_FP32, TX, TY, true, SCALAR>(I.fa[par], bx, by, local, sm);
            __syncthreads();     // shared memory is reused by the next item
        }
        ok = grid_sync(B);
        // diffusion sub-steps: sigma of the new buffer (par^1) and the old one as the other buffer
        for (int k = 0; k <= B.max_dsub && ok && n_dif > 0; ++k) {
            for (int item = blockIdx.x; item < n_dif; item += gridDim.x) {
                const int i = find_inst(B.dif_begin, B.n_inst, item);
                const BatchInst& I = B.inst[i];
                const int local = item - __ldg(B.dif_begin + i);
                const int by = local / I.dif_tx, bx = local - by * I.dif_tx;
                float* sn = I.sig[par ^ 1];
                float* so = I.sig[par];
                const long long NP = I.fa[0].plane;
                if (k < I.dsub) {
                    const bool even = (k & 1) == 0;
                    dif::diffuse_tile(even ? sn : so, even ? so : sn, NP, I.fa[0].nx, I.fa[0].ny, I.dsub_D, bx, by, sm);
                } else if (k == I.dsub && (I.dsub & 1)) {
                    // odd number of sub-steps: the result is in the other buffer; copy it back
                    for (int q = threadIdx.x; q < dif::DX * dif::DY; q += blockDim.x) {
                        const int ly = q / dif::DX, lx = q - ly * dif::DX;
                        const int gx = bx * dif::DX + lx, gy = by * dif::DY + ly;
                        if (gx < I.fa[0].nx && gy < I.fa[0].ny) {
                            const long long g = (long long)gy * I.fa[0].nx + gx;
                            for (int c = 0; c < 3; ++c) sn[c * NP + g] = __ldcg(so + c * NP + g);
                        }
                    }
                }
            }
            ok = grid_sync(B);
        }
        if (!ok) break;
        for (int item = blockIdx.x; item < n_nodes; item += gridDim.x) {
            const int i = find_inst(B.node_begin, B.n_inst, item);
            NodeArgs na = B.inst[i].na;
            na.X = B.inst[i].xb[par];
            na.X_out = B.inst[i].xb[par ^ 1];
            // the tiles' shared memory is free in this phase
            node::node_block(na, item - __ldg(B.node_begin + i), *reinterpret_cast<node::NodeSmem*>(sm));
            __syncthreads();
        }
        ok = grid_sync(B);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *B.cur = (cur0 + nsteps) & 1;
}

// ---- phase launches: one CTA per work item, the buffer parity of step s of the chunk read from
// the device word (so that a replayed graph continues from wherever the last chunk ended) ----

template <int TX, int TY, bool SCALAR>
__global__ void __launch_bounds__(BT, 3) k_batch_tiles(const BatchArgs B, int s)
{
    extern __shared__ __align__(16) float sm[];
    const int par = (*B.cur + s) & 1;
    const int item = blockIdx.x;
    const int i = find_inst(B.tile_begin, B.n_inst, item);
    const BatchInst& I = B.inst[i];
    const int local = item - __ldg(B.tile_begin + i);
    const int by = local / I.tiles_x, bx = local - by * I.tiles_x;
    // the state was written by an earlier launch: the read-only path is safe
    tile::tile_step<MODE_STEP, cell::PREC_FP32, TX, TY, false, SCALAR>(I.fa[par], bx, by, local, sm);
}

// the warp-strip step of every instance of the strip group: CTA `local` of an instance covers
// strip columns (local % tiles_x) * SWARPS .. and rows chunk local / tiles_x; the step index comes
// from the instance's control block (advanced by its node blocks of the step before)
template <bool SCALAR>
__global__ void __launch_bounds__(SNT, 3) k_batch_strips(const BatchArgs B, int s)
{
    extern __shared__ __align__(16) float smem[];
    const int par = (*B.cur + s) & 1;
    const int item = blockIdx.x;
    const int i = find_inst(B.tile_begin, B.n_inst, item);
    const BatchInst& I = B.inst[i];
    const int local = item - __ldg(B.tile_begin + i);
    const int cy = local / I.tiles_x, cx = local - cy * I.tiles_x;
    strip_body<cell::PREC_FP32, SCALAR>(I.fa[par], I.fa[par].ctl->t, STRIP_H, cx, cy, local, smem);
}

// sub-step k of the diffusion of the instances with dsub > k (or, with dsub odd and k == dsub,
// the copy of the result back into the new state's sigma planes)
__global__ void __launch_bounds__(BT) k_batch_diffuse(const BatchArgs B, int s, int k)
{
    extern __shared__ __align__(16) float sm[];
    const int par = (*B.cur + s) & 1;
    const int item = blockIdx.x;
    const int i = find_inst(B.dif_begin, B.n_inst, item);
    const BatchInst& I = B.inst[i];
    const int local = item - __ldg(B.dif_begin + i);
    const int by = local / I.dif_tx, bx = local - by * I.dif_tx;
    float* sn = I.sig[par ^ 1];
    float* so = I.sig[par];
    const long long NP = I.fa[0].plane;
    if (k < I.dsub) {
        const bool even = (k & 1) == 0;
        dif::diffuse_tile(even ? sn : so, even ? so : sn, NP, I.fa[0].nx, I.fa[0].ny, I.dsub_D, bx, by, sm);
    } else if (k == I.dsub && (I.dsub & 1)) {
        for (int q = threadIdx.x; q < dif::DX * dif::DY; q += blockDim.x) {
            const int ly = q / dif::DX, lx = q - ly * dif::DX;
            const int gx = bx * dif::DX + lx, gy = by * dif::DY + ly;
            if (gx < I.fa[0].nx && gy < I.fa[0].ny) {
                const long long g = (long long)gy * I.fa[0].nx + gx;
                for (int c = 0; c < 3; ++c) sn[c * NP + g] = so[c * NP + g];
            }
        }
    }
}

__global__ void __launch_bounds__(NODE_THREADS) k_batch_nodes(const BatchArgs B, int s)
{
    __shared__ node::NodeSmem S;
    const int par = (*B.cur + s) & 1;
    const int item = blockIdx.x;
    const int i = find_inst(B.node_begin, B.n_inst, item);
    NodeArgs na = B.inst[i].na;
    na.X = B.inst[i].xb[par];
    na.X_out = B.inst[i].xb[par ^ 1];
    node::node_block(na, item - __ldg(B.node_begin + i), S);
}

// the buffer parity after a chunk of n steps
__global__ void k_batch_parity(int* cur, int n)
{
    if (threadIdx.x == 0) *cur = (*cur + n) & 1;
}

}  // namespace
}  // namespace vlb

using namespace vlb;

struct lb_batch {
    std::vector<lb_handle*> h;
    cudaStream_t user = nullptr;            // the handles' stream
    cudaStream_t stream = nullptr;          // the batch's own stream (capturable)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    std::vector<int> shape;                 // per instance
    bool scalar = false;                    // every instance runs the scalar model (else none does)
    // per tile shape: the group of instances with that shape (device descriptors, prefix sums)
    BatchInst* d_inst[N_SHAPES] = {};
    int* d_tile_begin[N_SHAPES] = {};
    int* d_node_begin[N_SHAPES] = {};
    int* d_dif_begin[N_SHAPES] = {};
    int n_group[N_SHAPES] = {};
    int max_dsub[N_SHAPES] = {};
    int grid[N_SHAPES] = {};                // CTAs of each shape's persistent launch
    int n_tiles[N_SHAPES] = {};             // work items of each group (phase launches)
    int n_nodes[N_SHAPES] = {};
    int n_dif[N_SHAPES] = {};
    bool persistent = false;                // one persistent kernel per chunk (else phase launches)
    int* d_cur = nullptr;                   // buffer parity, one word per group
    unsigned* d_bar = nullptr;              // barrier words, two per group
    int* d_err = nullptr;
    std::vector<double*> partials;          // per instance: readout partial sums sized for any shape
    int chunk = 10;
    unsigned extra_arrivals = 0;
    unsigned long long wait_ns = 2000000000ull;
    cudaGraphExec_t graph = nullptr;
    bool graph_tried = false;
    std::string err;
};

namespace {

// the strip shape applies to this instance (the warp-strip kernel's conditions)
bool strip_ok(const lb_handle* h) { return strip_eligible(h->p.nx, h->p.ny, h->p.walls_x || h->p.walls_y); }

int bfail(lb_batch* b, int code, const std::string& msg)
{
    if (b) b->err = msg;
    return code;
}

#define BCK(b, call)                                                                   \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            if (b) b->err = std::string(#call) + ": " + cudaGetErrorString(e_);        \
            return e_ == cudaErrorMemoryAllocation ? LB_ENOMEM : LB_ECUDA;             \
        }                                                                              \
    } while (0)

void drop_graph(lb_batch* b)
{
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->graph_tried = false;
}

// (re)build the per-instance descriptors of every shape group for the current tile shapes
int build_plan(lb_batch* b)
{
    const int n = (int)b->h.size();
    for (int sh = 0; sh < N_SHAPES; ++sh) {
        std::vector<BatchInst> inst;
        std::vector<int> tb(1, 0), nb(1, 0), db(1, 0);
        b->max_dsub[sh] = 0;
        for (int i = 0; i < n; ++i) {
            if (b->shape[i] != sh) continue;
            lb_handle* h = b->h[i];
            BatchInst I;
            const int save = h->cur;
            for (int p = 0; p < 2; ++p) {
                h->cur = p;
                I.fa[p] = handle_fused_args(h);
                I.fa[p].partials = b->partials[i];
            }
            h->cur = save;
            I.na = handle_node_args(h, 1);
            I.na.partials = b->partials[i];
            I.xb[h->cur] = h->X;
            I.xb[h->cur ^ 1] = h->X_alt;
            I.shape = sh;
            if (sh == SHAPE_STRIP) {
                I.tiles_x = ((h->p.nx + SOWN - 1) / SOWN + SWARPS - 1) / SWARPS;
                I.tiles_y = (h->p.ny + STRIP_H - 1) / STRIP_H;
            } else {
                I.tiles_x = (h->p.nx + shape_tx(sh) - 1) / shape_tx(sh);
                I.tiles_y = (h->p.ny + shape_ty(sh) - 1) / shape_ty(sh);
            }
            I.na.n_partials = I.tiles_x * I.tiles_y;
            for (int p = 0; p < 2; ++p) I.sig[p] = static_cast<float*>(h->state[p]) + (size_t)PL_SXX * h->plane;
            I.dsub = h->p.diffusion_substeps;
            I.dsub_D = I.dsub > 0 ? (float)(h->p.Dp / I.dsub) : 0.f;
            I.dif_tx = diffuse_tiles_x(h->p.nx);
            I.dif_ty = diffuse_tiles_y(h->p.ny);
            b->max_dsub[sh] = std::max(b->max_dsub[sh], I.dsub);
            tb.push_back(tb.back() + I.tiles_x * I.tiles_y);
            nb.push_back(nb.back() + h->n_node_ctas);
            db.push_back(db.back() + (I.dsub > 0 ? I.dif_tx * I.dif_ty : 0));
            inst.push_back(I);
        }
        b->n_group[sh] = (int)inst.size();
        b->n_tiles[sh] = tb.back();
        b->n_nodes[sh] = nb.back();
        b->n_dif[sh] = db.back();
        if (inst.empty()) continue;
        const int g = (int)inst.size();
        BCK(b, cudaMemcpy(b->d_inst[sh], inst.data(), sizeof(BatchInst) * g, cudaMemcpyHostToDevice));
        BCK(b, cudaMemcpy(b->d_tile_begin[sh], tb.data(), sizeof(int) * (g + 1), cudaMemcpyHostToDevice));
        BCK(b, cudaMemcpy(b->d_node_begin[sh], nb.data(), sizeof(int) * (g + 1), cudaMemcpyHostToDevice));
        BCK(b, cudaMemcpy(b->d_dif_begin[sh], db.data(), sizeof(int) * (g + 1), cudaMemcpyHostToDevice));
    }
    drop_graph(b);
    return LB_OK;
}

BatchArgs batch_args(const lb_batch* b, int sh)
{
    BatchArgs a;
    a.inst = b->d_inst[sh];
    a.n_inst = b->n_group[sh];
    a.tile_begin = b->d_tile_begin[sh];
    a.node_begin = b->d_node_begin[sh];
    a.dif_begin = b->d_dif_begin[sh];
    a.max_dsub = b->max_dsub[sh];
    a.cur = b->d_cur + sh;
    a.bar = b->d_bar + 2 * sh;
    a.err = b->d_err;
    a.extra_arrivals = b->extra_arrivals;
    a.wait_ns = b->wait_ns;
    return a;
}

template <int TX, int TY>
cudaError_t launch_shape(const lb_batch* b, int sh, int nsteps)
{
    BatchArgs a = batch_args(b, sh);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(b->grid[sh]);
    cfg.blockDim = dim3(BT);
    cfg.dynamicSmemBytes = batch_smem<TX, TY>();
    cfg.stream = b->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return b->scalar ? cudaLaunchKernelEx(&cfg, k_batch<TX, TY, true>, a, nsteps)
                     : cudaLaunchKernelEx(&cfg, k_batch<TX, TY, false>, a, nsteps);
}

template <int TX, int TY>
cudaError_t launch_tiles(const lb_batch* b, int sh, int s)
{
    static unsigned long long attr_done = 0;     // per device
    auto kern = b->scalar ? k_batch_tiles<TX, TY, true> : k_batch_tiles<TX, TY, false>;
    const size_t smem = tile::TileGeo<TX, TY>::SMEM_BYTES;
    if (!done_on_device(attr_done)) {
        cudaError_t e = cudaFuncSetAttribute(k_batch_tiles<TX, TY, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_batch_tiles<TX, TY, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) {
            attr_done = 0;
            return e;
        }
    }
    kern<<<b->n_tiles[sh], BT, smem, b->stream>>>(batch_args(b, sh), s);
    return cudaGetLastError();
}

cudaError_t launch_strips(const lb_batch* b, int s)
{
    static unsigned long long attr_done = 0;     // per device
    if (!done_on_device(attr_done)) {
        cudaError_t e = cudaFuncSetAttribute(k_batch_strips<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)STRIP_SMEM);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_batch_strips<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)STRIP_SMEM);
        if (e != cudaSuccess) {
            attr_done = 0;
            return e;
        }
    }
    auto kern = b->scalar ? k_batch_strips<true> : k_batch_strips<false>;
    kern<<<b->n_tiles[SHAPE_STRIP], SNT, STRIP_SMEM, b->stream>>>(batch_args(b, SHAPE_STRIP), s);
    return cudaGetLastError();
}

// Phase launches of `nsteps` steps: per step the lattice tiles of every group, then the
// diffusion sub-steps, then the node blocks; at the end the device parity words advance.
cudaError_t launch_phases(const lb_batch* b, int nsteps)
{
    cudaError_t e = cudaSuccess;
    const size_t dsm = sizeof(float) * dif::SMEM;
    for (int s = 0; s < nsteps && e == cudaSuccess; ++s) {
        if (b->n_group[0] && e == cudaSuccess) e = launch_tiles<32, 16>(b, 0, s);
        if (b->n_group[1] && e == cudaSuccess) e = launch_tiles<32, 8>(b, 1, s);
        if (b->n_group[2] && e == cudaSuccess) e = launch_tiles<64, 8>(b, 2, s);
        if (b->n_group[3] && e == cudaSuccess) e = launch_tiles<16, 16>(b, 3, s);
        if (b->n_group[SHAPE_STRIP] && e == cudaSuccess) e = launch_strips(b, s);
        for (int sh = 0; sh < N_SHAPES && e == cudaSuccess; ++sh) {
            if (!b->n_group[sh] || !b->n_dif[sh]) continue;
            for (int k = 0; k <= b->max_dsub[sh] && e == cudaSuccess; ++k) {
                k_batch_diffuse<<<b->n_dif[sh], BT, dsm, b->stream>>>(batch_args(b, sh), s, k);
                e = cudaGetLastError();
            }
        }
        for (int sh = 0; sh < N_SHAPES && e == cudaSuccess; ++sh) {
            if (!b->n_group[sh] || !b->n_nodes[sh]) continue;
            k_batch_nodes<<<b->n_nodes[sh], NODE_THREADS, 0, b->stream>>>(batch_args(b, sh), s);
            e = cudaGetLastError();
        }
    }
    for (int sh = 0; sh < N_SHAPES && e == cudaSuccess; ++sh) {
        if (!b->n_group[sh]) continue;
        k_batch_parity<<<1, 32, 0, b->stream>>>(b->d_cur + sh, nsteps);
        e = cudaGetLastError();
    }
    return e;
}

// one persistent launch per non-empty shape group, one after another on the batch stream (or
// the phase launches)
cudaError_t launch_batch(const lb_batch* b, int nsteps)
{
    if (!b->persistent) return launch_phases(b, nsteps);
    cudaError_t e = cudaSuccess;
    if (b->n_group[0] && e == cudaSuccess) e = launch_shape<32, 16>(b, 0, nsteps);
    if (b->n_group[1] && e == cudaSuccess) e = launch_shape<32, 8>(b, 1, nsteps);
    if (b->n_group[2] && e == cudaSuccess) e = launch_shape<64, 8>(b, 2, nsteps);
    if (b->n_group[3] && e == cudaSuccess) e = launch_shape<16, 16>(b, 3, nsteps);
    return e;
}

// shared-memory opt-in and the co-resident grid of one shape's kernel
template <int TX, int TY>
cudaError_t setup_shape(lb_batch* b, int sh, int n_sm)
{
    const size_t smem = batch_smem<TX, TY>();
    auto kern = b->scalar ? k_batch<TX, TY, true> : k_batch<TX, TY, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BT, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    b->grid[sh] = n_sm * per_sm;
    return cudaSuccess;
}

// Capture one persistent launch of `chunk` steps as a graph (once per plan).  If capture or
// instantiation is refused, the batch keeps launching the kernel directly.
void capture(lb_batch* b)
{
    b->graph_tried = true;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    const cudaError_t e = launch_batch(b, b->chunk);
    const cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (e == cudaSuccess && e2 == cudaSuccess && g && cudaGraphInstantiate(&b->graph, g, 0) != cudaSuccess)
        b->graph = nullptr;
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
}

// n steps on the batch stream, ordered after the work already queued on the handles' stream and
// before anything queued there later
int run_steps(lb_batch* b, long long n)
{
    if (n == 0) return LB_OK;
    if (!b->graph_tried) capture(b);
    BCK(b, cudaEventRecord(b->ev_in, b->user));
    BCK(b, cudaStreamWaitEvent(b->stream, b->ev_in, 0));
    long long left = n;
    while (b->graph && left >= b->chunk) {
        BCK(b, cudaGraphLaunch(b->graph, b->stream));
        left -= b->chunk;
    }
    while (left > 0) {
        const int k = (int)std::min<long long>(left, b->chunk);
        BCK(b, launch_batch(b, k));
        left -= k;
    }
    BCK(b, cudaEventRecord(b->ev_out, b->stream));
    BCK(b, cudaStreamWaitEvent(b->user, b->ev_out, 0));
    for (lb_handle* h : b->h) {
        h->t += n;
        h->cur ^= (int)(n & 1);
        if (n & 1) std::swap(h->X, h->X_alt);
    }
    return LB_OK;
}

}  // namespace

extern "C" {

int lb_batch_create(lb_handle* const* handles, int32_t n, lb_batch** out)
{
    if (!handles || n < 1 || !out) return LB_EINVAL;
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        const lb_handle* h = handles[i];
        if (!h || !h->fields_ready || !h->node_work) return LB_ESTATE;
        if (h->p.precision != LB_FP32 || h->p.model != handles[0]->p.model || h->cur != handles[0]->cur ||
            h->stream != handles[0]->stream)
            return LB_EINVAL;
        for (int k = 0; k < i; ++k)
            if (handles[k] == h) return LB_EINVAL;
    }
    lb_batch* b = new lb_batch();
    b->h.assign(handles, handles + n);
    for (lb_handle* h : b->h) ++h->batch_refs;   // its graphs hold the handles' state buffers
    b->user = handles[0]->stream;
    b->chunk = std::max(1, handles[0]->p.readout_every);
    b->shape.assign(n, 0);
    b->scalar = handles[0]->p.model == LB_MODEL_SCALAR;
    auto cleanup = [&](int code) { lb_batch_destroy(b); return code; };
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) != cudaSuccess)
        return cleanup(LB_ECUDA);
    for (int sh = 0; sh < N_SHAPES; ++sh)
        if (cudaMalloc(&b->d_inst[sh], sizeof(BatchInst) * n) != cudaSuccess ||
            cudaMalloc(&b->d_tile_begin[sh], sizeof(int) * (n + 1)) != cudaSuccess ||
            cudaMalloc(&b->d_node_begin[sh], sizeof(int) * (n + 1)) != cudaSuccess ||
            cudaMalloc(&b->d_dif_begin[sh], sizeof(int) * (n + 1)) != cudaSuccess)
            return cleanup(LB_ENOMEM);
    if (cudaMalloc(&b->d_cur, sizeof(int) * N_SHAPES) != cudaSuccess ||
        cudaMalloc(&b->d_bar, 2 * sizeof(unsigned) * N_SHAPES) != cudaSuccess ||
        cudaMalloc(&b->d_err, sizeof(int)) != cudaSuccess)
        return cleanup(LB_ENOMEM);
    for (int i = 0; i < n; ++i) {
        // enough partial sums for the smallest tile (16 x 8 cells covers every shape's count)
        double* p = nullptr;
        const long long tiles = ((long long)b->h[i]->p.nx / 16 + 1) * ((long long)b->h[i]->p.ny / 8 + 1);
        if (cudaMalloc(&p, sizeof(double) * 5 * tiles) != cudaSuccess) return cleanup(LB_ENOMEM);
        b->partials.push_back(p);
    }
    // the handles' queued work must be done before the batch's control words are set
    if (cudaStreamSynchronize(b->user) != cudaSuccess) return cleanup(LB_ECUDA);
    const int c0 = handles[0]->cur;
    const int c4[N_SHAPES] = {c0, c0, c0, c0};
    if (cudaMemcpy(b->d_cur, c4, sizeof(c4), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(b->d_bar, 0, 2 * sizeof(unsigned) * N_SHAPES) != cudaSuccess ||
        cudaMemset(b->d_err, 0, sizeof(int)) != cudaSuccess)
        return cleanup(LB_ECUDA);
    int dev = 0, n_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (setup_shape<32, 16>(b, 0, n_sm) != cudaSuccess || setup_shape<32, 8>(b, 1, n_sm) != cudaSuccess ||
        setup_shape<64, 8>(b, 2, n_sm) != cudaSuccess || setup_shape<16, 16>(b, 3, n_sm) != cudaSuccess)
        return cleanup(LB_ECUDA);
    const int rc = build_plan(b);
    if (rc != LB_OK) return cleanup(rc);
    *out = b;
    return LB_OK;
}

int lb_batch_set_shape(lb_batch* b, int32_t inst, int32_t shape)
{
    if (!b) return LB_EINVAL;
    if (inst < -1 || inst >= (int)b->h.size() || shape < 0 || shape >= N_SHAPES)
        return bfail(b, LB_EINVAL, "bad instance or shape");
    if (shape == SHAPE_STRIP) {
        if (b->persistent) return bfail(b, LB_EINVAL, "the strip shape runs with phase launches only");
        for (int i = 0; i < (int)b->h.size(); ++i)
            if ((inst < 0 || i == inst) && !strip_ok(b->h[i]))
                return bfail(b, LB_EINVAL, "instance " + std::to_string(i) + " cannot take the strip shape "
                             "(periodic, nx >= 64 even, ny >= 32)");
    }
    BCK(b, cudaStreamSynchronize(b->stream));
    if (inst < 0) std::fill(b->shape.begin(), b->shape.end(), shape);
    else b->shape[inst] = shape;
    return build_plan(b);
}

int32_t lb_batch_shape(const lb_batch* b, int32_t inst)
{
    return b && inst >= 0 && inst < (int)b->h.size() ? b->shape[inst] : -1;
}

int lb_batch_step(lb_batch* b, int64_t n)
{
    if (!b) return LB_EINVAL;
    if (n < 0) return bfail(b, LB_EINVAL, "n < 0");
    return run_steps(b, n);
}

int lb_batch_sync(lb_batch* b)
{
    if (!b) return LB_EINVAL;
    BCK(b, cudaStreamSynchronize(b->stream));
    BCK(b, cudaStreamSynchronize(b->user));
    int e = 0;
    BCK(b, cudaMemcpy(&e, b->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) {
        const int z = 0;
        unsigned zb[2 * N_SHAPES] = {};
        BCK(b, cudaMemcpy(b->d_err, &z, sizeof(int), cudaMemcpyHostToDevice));
        BCK(b, cudaMemcpy(b->d_bar, zb, sizeof zb, cudaMemcpyHostToDevice));
        return bfail(b, LB_ETIMEOUT, "a grid barrier of the batched kernel timed out; the states are undefined");
    }
    for (size_t i = 0; i < b->h.size(); ++i) {
        const int rc = lb_sync(b->h[i]);
        if (rc != LB_OK) return bfail(b, rc, "instance " + std::to_string(i) + ": " + lb_last_error(b->h[i]));
    }
    return LB_OK;
}

int32_t lb_batch_grid(const lb_batch* b)
{
    if (!b) return 0;
    if (b->persistent) return b->grid[0];
    int n = 0;
    for (int sh = 0; sh < N_SHAPES; ++sh) n += b->n_group[sh] ? b->n_tiles[sh] : 0;
    return n;
}

int lb_batch_set_persistent(lb_batch* b, int32_t enable)
{
    if (!b) return LB_EINVAL;
    if (enable != 0 && enable != 1) return bfail(b, LB_EINVAL, "enable must be 0 or 1");
    BCK(b, cudaStreamSynchronize(b->stream));
    if (enable)
        for (int sh : b->shape)
            if (sh == SHAPE_STRIP) return bfail(b, LB_EINVAL, "an instance has the strip shape (phase launches only)");
    b->persistent = enable != 0;
    drop_graph(b);
    return LB_OK;
}

int32_t lb_batch_uses_graph(const lb_batch* b) { return b && b->graph ? 1 : 0; }

int lb_batch_set_wait_limit(lb_batch* b, double wait_ms, int32_t extra_arrivals)
{
    if (!b) return LB_EINVAL;
    if (!(wait_ms > 0.0 && wait_ms <= 60000.0) || extra_arrivals < 0)
        return bfail(b, LB_EINVAL, "need 0 < wait_ms <= 60000 and extra_arrivals >= 0");
    BCK(b, cudaStreamSynchronize(b->stream));
    b->wait_ns = (unsigned long long)(wait_ms * 1e6);
    b->extra_arrivals = (unsigned)extra_arrivals;
    drop_graph(b);
    return LB_OK;
}

// Autotuner: for every distinct lattice size of the batch, time `steps` batch steps with each
// tile shape applied to that size (the others unchanged) and keep the fastest.  The state is
// saved before and restored after, so tuning does not advance the simulation.  With a cache
// path, sizes already tuned on this GPU model are read from it and new results written back.
int lb_batch_autotune(lb_batch* b, const char* cache_path, int32_t steps)
{
    if (!b) return LB_EINVAL;
    if (steps < 1) return bfail(b, LB_EINVAL, "steps < 1");
    BCK(b, cudaStreamSynchronize(b->user));
    BCK(b, cudaStreamSynchronize(b->stream));
    cudaDeviceProp prop;
    int dev = 0;
    BCK(b, cudaGetDevice(&dev));
    BCK(b, cudaGetDeviceProperties(&prop, dev));
    std::map<std::string, int> cache;
    if (cache_path) {
        // flat JSON object, one entry per line:  "<gpu>|<nx>x<ny>": <shape>
        if (FILE* f = fopen(cache_path, "r")) {
            char line[512];
            while (fgets(line, sizeof line, f)) {
                char* q1 = strchr(line, '"');
                char* q2 = q1 ? strchr(q1 + 1, '"') : nullptr;
                int v = -1;
                if (q1 && q2 && sscanf(q2 + 1, " : %d", &v) == 1 && v >= 0 && v < N_SHAPES)
                    cache[std::string(q1 + 1, q2)] = v;
            }
            fclose(f);
        }
    }
    auto key_of = [&](const lb_handle* h) {
        return std::string(prop.name) + "|" + std::to_string(h->p.nx) + "x" + std::to_string(h->p.ny);
    };
    std::map<std::string, std::vector<int>> classes;
    for (int i = 0; i < (int)b->h.size(); ++i) classes[key_of(b->h[i])].push_back(i);
    bool need_tune = false;
    for (auto& kv : classes)
        if (!cache.count(kv.first)) need_tune = true;
    // snapshot everything a step writes: both state buffers, control words, series, nodes, rings
    std::vector<std::pair<void*, void*>> saved;      // (live, copy)
    std::vector<size_t> saved_bytes;
    auto release = [&]() {
        for (auto& s : saved) cudaFree(s.second);
        saved.clear();
    };
    if (need_tune) {
        for (lb_handle* h : b->h) {
            const size_t sb = (size_t)h->esz * N_PLANES * h->plane;
            std::vector<std::pair<void*, size_t>> items = {
                {h->state[0], sb}, {h->state[1], sb}, {h->ctl, sizeof(Ctl)},
                {h->series, sizeof(double) * (size_t)h->series_cap * h->row_len}};
            if (h->n_total > 0) {
                items.push_back({h->X, sizeof(double2) * h->n_total});
                items.push_back({h->node_cell, sizeof(int2) * h->n_total});
                items.push_back({h->node_frac, sizeof(float2) * h->n_total});
                items.push_back({h->node_force, sizeof(float2) * h->n_total});
                items.push_back({h->rings, sizeof(RingDev) * h->n_rings});
            }
            for (auto& it : items) {
                void* d = nullptr;
                if (cudaMalloc(&d, it.second) != cudaSuccess) {
                    release();
                    return bfail(b, LB_ENOMEM, "autotune snapshot");
                }
                saved.push_back({it.first, d});
                saved_bytes.push_back(it.second);
                if (cudaMemcpy(d, it.first, it.second, cudaMemcpyDeviceToDevice) != cudaSuccess) {
                    release();
                    return bfail(b, LB_ECUDA, "autotune snapshot copy");
                }
            }
        }
    }
    int dcur[N_SHAPES] = {};
    BCK(b, cudaMemcpy(dcur, b->d_cur, sizeof dcur, cudaMemcpyDeviceToHost));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int rc = LB_OK;
    // time `steps` batch steps with the current shapes (after one warm-up step); < 0 on error
    auto time_plan = [&]() -> float {
        if ((rc = build_plan(b)) != LB_OK) return -1.f;
        cudaError_t e = launch_batch(b, 1);
        if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
        if (e == cudaSuccess) e = launch_batch(b, steps);
        if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            rc = bfail(b, LB_ECUDA, std::string("autotune launch: ") + cudaGetErrorString(e));
            return -1.f;
        }
        return ms;
    };
    auto allowed = [&](int sh, int i) { return sh != SHAPE_STRIP || (!b->persistent && strip_ok(b->h[i])); };
    // First one shape for every untuned instance (one launch per phase for the whole batch: a
    // shape can pay only when most of the batch takes it), then each size class on its own from
    // there, the other classes fixed.
    if (need_tune) {
        float best = 3.0e38f;
        int best_s = 0;
        for (int sh = 0; sh < N_SHAPES && rc == LB_OK; ++sh) {
            bool ok = true;
            for (auto& kv : classes)
                if (!cache.count(kv.first))
                    for (int i : kv.second) ok = ok && allowed(sh, i);
            if (!ok) continue;
            for (auto& kv : classes) {
                auto hit = cache.find(kv.first);
                for (int i : kv.second) b->shape[i] = hit != cache.end() ? hit->second : sh;
            }
            const float ms = time_plan();
            if (ms >= 0.f && ms < best) {
                best = ms;
                best_s = sh;
            }
        }
        for (auto& kv : classes)
            if (!cache.count(kv.first))
                for (int i : kv.second) b->shape[i] = best_s;
    }
    for (auto& kv : classes) {
        if (rc != LB_OK) break;
        auto hit = cache.find(kv.first);
        if (hit != cache.end()) {
            for (int i : kv.second) b->shape[i] = hit->second;
            continue;
        }
        const int start = b->shape[kv.second[0]];
        float best = time_plan();
        int best_s = start;
        for (int sh = 0; sh < N_SHAPES && rc == LB_OK; ++sh) {
            if (sh == start || !allowed(sh, kv.second[0])) continue;
            for (int i : kv.second) b->shape[i] = sh;
            const float ms = time_plan();
            if (ms >= 0.f && ms < best) {
                best = ms;
                best_s = sh;
            }
        }
        for (int i : kv.second) b->shape[i] = best_s;
        cache[kv.first] = best_s;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // restore the states, the device parity and the barrier words
    for (size_t k = 0; k < saved.size(); ++k)
        cudaMemcpy(saved[k].first, saved[k].second, saved_bytes[k], cudaMemcpyDeviceToDevice);
    release();
    cudaMemcpy(b->d_cur, dcur, sizeof dcur, cudaMemcpyHostToDevice);
    int berr = 0;
    cudaMemcpy(&berr, b->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (rc != LB_OK) return rc;
    if (berr) return bfail(b, LB_ETIMEOUT, "a grid barrier timed out while tuning");
    rc = build_plan(b);
    if (rc != LB_OK) return rc;
    if (cache_path && need_tune) {
        if (FILE* f = fopen(cache_path, "w")) {
            fprintf(f, "{\n");
            size_t k = 0;
            for (auto& kv : cache)
                fprintf(f, "  \"%s\": %d%s\n", kv.first.c_str(), kv.second, ++k < cache.size() ? "," : "");
            fprintf(f, "}\n");
            fclose(f);
        } else {
            return bfail(b, LB_EINVAL, std::string("cannot write the tuning cache ") + cache_path);
        }
    }
    return LB_OK;
}

const char* lb_batch_last_error(const lb_batch* b) { return b ? b->err.c_str() : "null batch"; }

void lb_batch_destroy(lb_batch* b)
{
    if (!b) return;
    for (lb_handle* h : b->h) --h->batch_refs;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->stream) cudaStreamDestroy(b->stream);
    for (int sh = 0; sh < N_SHAPES; ++sh) {
        cudaFree(b->d_inst[sh]);
        cudaFree(b->d_tile_begin[sh]);
        cudaFree(b->d_node_begin[sh]);
        cudaFree(b->d_dif_begin[sh]);
    }
    cudaFree(b->d_cur);
    cudaFree(b->d_bar);
    cudaFree(b->d_err);
    for (double* p : b->partials) cudaFree(p);
    delete b;
}

}  // extern "C"
