// lb_fused.cu -- the tile kernels: one CTA per 32 x 16 tile of the fused step (lb_tile.cuh), one
// cell per thread (tile_step) or two neighbouring cells per thread on paired FP32 instructions
// (tile_step2); optionally with the node step of the same time step in their tail.
#include <cuda_runtime.h>

#include <cmath>

#include "lb_node.cuh"
#include "lb_tile.cuh"

namespace vlb {

namespace {

using namespace tile;

// Tiles c = 0 .. n_tiles - 1 of one lattice axis whose staged region [c T - 2, c T - 2 + RW)
// meets the box span [b, b + bw) (the test of ib_gather); one warp, result in every lane.
__device__ __forceinline__ int tiles_meeting(int n_tiles, int T, int RW, int b, int bw, int n)
{
    const int lane = threadIdx.x & 31;
    int cnt = 0;
    for (int c0 = 0; c0 < n_tiles; c0 += 32) {
        const int c = c0 + lane;
        cnt += __popc(__ballot_sync(0xffffffffu, c < n_tiles && meets(c * T - 2, RW, b, bw, n)));
    }
    return cnt;
}

// One open node block of a ring at step tag (t + 1): increments the claim count of
// ring_claim (tag << 16 | count) while it is below nc and returns the claimed block, or -1.
// Each failed exchange means another CTA claimed a block, so at most nc + 1 rounds run; the
// bound only guards that argument.
__device__ __forceinline__ int claim_block(unsigned long long* p, unsigned long long tag, int nc, int* err)
{
    unsigned long long w = __ldcg(p);
    for (int it = 0; it < 4096; ++it) {
        if ((w >> 16) != tag || (int)(w & 0xffffu) >= nc) return -1;
        const unsigned long long old = atomicCAS(p, w, w + 1);
        if (old == w) return (int)(w & 0xffffu);
        w = old;
    }
    atomicExch(err, 1);
    return -1;
}

// Node blocks of the rings in `open` (bits; ring r0 + bit), claimed one at a time, then (last)
// the lattice readout sums: the rare parts of the node tail, kept out of line so that the tiles
// that have none of it pay nothing for them.  The node blocks take the tile's shared memory,
// whose staged fields are dead once every thread has passed the barrier at the start.
__device__ __noinline__ void tail_work(const FusedArgs& a, unsigned open, int r0, bool last, float* sm)
{
    node::NodeSmem& S = *reinterpret_cast<node::NodeSmem*>(sm);
    const int tid = threadIdx.x;
    const long long t = a.t;
    const unsigned long long tag = (unsigned long long)(t + 1);
    __syncthreads();
    while (open) {
        const int r = r0 + __ffs(open) - 1;
        open &= open - 1;
        const int c0 = a.na.ring_cta0[r], nc = a.na.ring_ctas[r];
        for (;;) {
            __syncthreads();
            if (tid == 0) S.flag[0] = claim_block(a.ring_claim + r, tag, nc, &a.ctl->err_timeout);
            __syncthreads();
            const int c = S.flag[0];
            if (c < 0) break;
            __threadfence();
            node::node_block(a.na, c0 + c, S, false, t);
        }
    }
    if (last) {
        __syncthreads();
        __threadfence();
        if (tid == 0) a.ctl->tile_ticket = 0u;
        node::lattice_readout(a.na, t, S.dred);
    }
}

// tiles that look for open node blocks in their tail: one in 32 in launch order, and all of the
// last thirty-second (rings whose tiles run late still find helpers)
__device__ __forceinline__ bool helper_tile()
{
    const int order = blockIdx.y * gridDim.x + blockIdx.x, total = gridDim.x * gridDim.y;
    return (order & 31) == 0 || order >= total - total / 32;
}

// The node step in the tail of the lattice kernel (FusedArgs::node_tail), after this tile's
// step (App. A).  A ring's nodes are read (spreading) only by the tiles whose region meets its
// box of step t, and the node update writes only the box of step t + 1 (RingDev::box), the
// nodes and the other position buffer: so once the last of those tiles has written u(t) and
// f^p(t) onto the box, the ring can advance while the remaining tiles run.  That tile opens the
// ring's node blocks; it and the helper tiles that finish later (helper_tile, and any tile that
// met a ring) run them, one claimed block at a time.  On readout steps every tile counts itself
// and the last one sums the lattice readout.  Flags live in the scan scratch of ib_gather (free
// by now; the ring masks after it stay intact).  Out of line: node_tail below calls it only for
// the tiles that have something to do.
template <int TX, int TY>
__device__ __noinline__ void node_tail_work(const FusedArgs& a, float* sm)
{
    using G = TileGeo<TX, TY>;
    static_assert(sizeof(node::NodeSmem) <= sizeof(float) * G::OFF_SC, "node blocks overlay the staged fields only");
    int* sT = reinterpret_cast<int*>(sm + G::OFF_SC);
    const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
    const int nr = a.n_rings;
    const long long t = a.t;
    const int bx = blockIdx.x;
    int by = blockIdx.y + a.tile_rot;
    if (by >= (int)gridDim.y) by -= gridDim.y;
    bool helper = helper_tile();
    const bool readout = (t % a.every) == 0;
    const unsigned meet = nr > 32 ? 0xffffffffu : (unsigned)sT[NT / 32 + 2];
    const unsigned long long tag = (unsigned long long)(t + 1);
    // the CTA's global writes of the step (state, boxes, partials) before any of its arrivals
    __threadfence();
    for (int r = 0; r < nr && meet != 0u; ++r) {
        if (nr <= 32 && !((meet >> r) & 1u)) continue;
        const int4 B = ring_box(a.rings[r], t);
        if (nr > 32 &&
            (!meets(bx * TX - 2, G::R2W, B.x, B.z, a.nx) || !meets(by * TY - 2, G::R2H, B.y, B.w, a.ny)))
            continue;
        helper = true;
        if (wid == 0) {
            const int c = tiles_meeting(gridDim.x, TX, G::R2W, B.x, B.z, a.nx);
            if (lane == 0) sT[0] = c;
        } else if (wid == 1) {
            const int c = tiles_meeting(gridDim.y, TY, G::R2H, B.y, B.w, a.ny);
            if (lane == 0) sT[1] = c;
        }
        __syncthreads();
        if (tid == 0) {
            const unsigned prev = atomicAdd(&a.box_tickets[r], 1u);
            if (prev == (unsigned)(sT[0] * sT[1] - 1)) {
                // every tile meeting the box is done with it: open the ring's node blocks
                a.box_tickets[r] = 0u;
                __threadfence();
                atomicExch(&a.ring_claim[r], tag << 16);
            }
        }
        __syncthreads();
    }
    // open node blocks of any ring (helpers), 32 rings at a time
    for (int r0 = 0; r0 < (helper ? nr : 0); r0 += 32) {
        if (wid == 0) {
            const int r = r0 + lane;
            bool open = false;
            if (r < nr) {
                const unsigned long long w = __ldcg(a.ring_claim + r);
                open = (w >> 16) == tag && (int)(w & 0xffffu) < a.na.ring_ctas[r];
            }
            const unsigned m = __ballot_sync(0xffffffffu, open);
            if (lane == 0) sT[2] = (int)m;
        }
        __syncthreads();
        const unsigned m = (unsigned)sT[2];
        if (m) tail_work(a, m, r0, false, sm);
        __syncthreads();
    }
    if (readout) {
        // every tile counts itself; the last one sums the lattice readout
        __syncthreads();
        if (tid == 0) sT[3] = atomicAdd(&a.ctl->tile_ticket, 1u) == gridDim.x * gridDim.y - 1u;
        __syncthreads();
        if (sT[3]) tail_work(a, 0u, 0, true, sm);
    }
}

// The node tail of one tile: the step counter (one tile), then node_tail_work where this tile
// meets a ring's box, is a helper, or the step is a readout step; nothing else for most tiles.
template <int TX, int TY>
__device__ __forceinline__ void node_tail(const FusedArgs& a, float* sm)
{
    using G = TileGeo<TX, TY>;
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) a.ctl->t = a.t + 1;   // nothing here reads it
    const int* sT = reinterpret_cast<const int*>(sm + G::OFF_SC);
    // the rings whose box meets this tile's staged region (tested in ib_gather for up to 32 rings)
    if (a.n_rings > 32 || sT[NT / 32 + 2] != 0 || helper_tile() || (a.t % a.every) == 0)
        node_tail_work<TX, TY>(a, sm);
}

template <int MODE, int PREC, bool SCALAR = false>
__global__ void __launch_bounds__(NT, 3) k_fused(const FusedArgs a)
{
    extern __shared__ __align__(16) float sm[];
    const bool tail = MODE == MODE_STEP && a.node_tail;
    int by = blockIdx.y;
    if (tail) {
        // consecutive lattice launches: the state staged first was written by the previous one
        pdl_wait();
        by += a.tile_rot;
        if (by >= (int)gridDim.y) by -= gridDim.y;
    }
    tile_step<MODE, PREC, TILE_X, TILE_Y, false, SCALAR>(a, blockIdx.x, by, by * gridDim.x + blockIdx.x, sm);
    if (tail) node_tail<TILE_X, TILE_Y>(a, sm);
}

template <int MODE, int PREC>
__global__ void __launch_bounds__(NT, 2) k_fused_pair(const FusedArgs a)
{
    extern __shared__ __align__(16) float sm[];
    const bool tail = MODE == MODE_STEP && a.node_tail;
    int by = blockIdx.y;
    if (tail) {
        pdl_wait();
        by += a.tile_rot;
        if (by >= (int)gridDim.y) by -= gridDim.y;
    }
    tile_step2<MODE, PREC, TILE_X, TILE_Y>(a, blockIdx.x, by, by * gridDim.x + blockIdx.x, sm);
    if (tail) node_tail<TILE_X, TILE_Y>(a, sm);
}

}  // namespace

int fused_ctas(int nx, int ny) { return ((nx + TILE_X - 1) / TILE_X) * ((ny + TILE_Y - 1) / TILE_Y); }

int fused_tile_rot(int nx, int ny, double y_top)
{
    (void)nx;
    const int ty = (ny + TILE_Y - 1) / TILE_Y;
    int row = (int)std::floor(y_top / TILE_Y) % ty;
    if (row < 0) row += ty;
    return row;
}

template <int MODE, int PREC, bool PAIR, bool SCALAR = false>
static cudaError_t launch_one(const FusedArgs& a, dim3 grid, cudaStream_t s, bool pdl)
{
    static unsigned long long attr_done = 0;     // per device
    auto kern = PAIR ? k_fused_pair<MODE, PREC> : k_fused<MODE, PREC, SCALAR>;
    if (!done_on_device(attr_done)) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)TileGeo<TILE_X, TILE_Y>::SMEM_BYTES);
        if (e != cudaSuccess) {
            attr_done = 0;
            return e;
        }
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = TileGeo<TILE_X, TILE_Y>::SMEM_BYTES;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, a);
}

template <bool PAIR>
static cudaError_t launch_form(const FusedArgs& a, int mode, dim3 grid, cudaStream_t s, bool pdl)
{
    // the scalar model's step (FP32 state, one-cell tiles); its moments pass is the tensorial one,
    // which reads the unchanged P planes and, with the Ericksen force off, does not use them
    if (!PAIR && a.scalar && a.prec == PREC_FP32 && mode == MODE_STEP)
        return launch_one<MODE_STEP, PREC_FP32, false, true>(a, grid, s, pdl);
    if (a.prec == PREC_FP32)
        return mode == MODE_STEP ? launch_one<MODE_STEP, PREC_FP32, PAIR>(a, grid, s, pdl)
                                 : launch_one<MODE_MOMENTS, PREC_FP32, PAIR>(a, grid, s, false);
    return mode == MODE_STEP ? launch_one<MODE_STEP, PREC_LP, PAIR>(a, grid, s, pdl)
                             : launch_one<MODE_MOMENTS, PREC_LP, PAIR>(a, grid, s, false);
}

cudaError_t launch_fused(const FusedArgs& a, int mode, cudaStream_t s, int* grid_ctas, bool pdl, bool pair)
{
    dim3 grid((a.nx + TILE_X - 1) / TILE_X, (a.ny + TILE_Y - 1) / TILE_Y);
    if (grid_ctas) *grid_ctas = grid.x * grid.y;
    return pair ? launch_form<true>(a, mode, grid, s, pdl) : launch_form<false>(a, mode, grid, s, pdl);
}

}  // namespace vlb
