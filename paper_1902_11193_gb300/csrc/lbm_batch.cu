// Batched parameter sweep: many lattices stepped by one persistent kernel.
//
// The paper's study (Secs. 4.1-4.3) runs the same solver over Sets A-E, a
// tau sweep and several geometries and resolutions.  Small lattices are
// launch-bound when stepped one by one, so the batch flattens every active
// lattice into a table of 256*npt-unit tiles and a persistent cooperative
// kernel walks the table once per time step, with a grid barrier between
// steps (each lattice's AA step t+1 reads what step t wrote).  The barrier
// waits are bounded in time: on expiry the kernel raises an error flag and
// returns, and the host reports LBM_ETIMEOUT.  In the last two steps of a
// chunk (three under the two-step-mean rule) every 256-unit group of a tile
// reduces its shifted velocity into an FP64 partial exactly as a
// single-lattice block does, a per-lattice kernel sums the partials in the
// single-lattice finalize's order, and the host applies each lattice's
// stopping rule and retires converged lattices from the table.
// The chunk (step-count upload, persistent kernel, reductions, result copy)
// is captured once in a CUDA graph and replayed; the tile table lives in
// device memory, so retiring lattices does not change the graph.
// Every lattice is an ordinary lbm_ctx (its own populations and link
// tables), so all single-lattice readers work on batch members, and the
// per-unit update is the same code as the single-lattice kernels
// (lbm_step.cuh) with the same explicitly rounded collision: a batch
// member's state, step count and measured mean velocity are bitwise those of
// the same lattice run alone with the same check interval and the default
// 256-thread blocks.
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "lbm_step.cuh"

namespace lbm {

SparseMap sparse_map(const lbm_ctx *c);
int launch_step(lbm_ctx *c, bool reduce);
int enqueue_measured_chunk(lbm_ctx *c, int64_t plain, int nmeas);

struct BatchLat {
    int layout;  // LBM_LAYOUT_AA or LBM_LAYOUT_SPARSE
    int npt;     // units per thread per tile (persistent kernel)
    uint32_t units;
    uint32_t goff;  // first of the lattice's 256-unit groups in the stepwise partials
    void *pop;
    const uint32_t *lw;
    SparseMap sm;
    Dims d;
    Collide<float> pf;  // collision parameters, built like the single-lattice ones
    Collide<double> pd;
    double inv_N;
};

template <typename C>
__device__ __forceinline__ const Collide<C> &lat_params(const BatchLat &L);
template <>
__device__ __forceinline__ const Collide<float> &lat_params<float>(const BatchLat &L) { return L.pf; }
template <>
__device__ __forceinline__ const Collide<double> &lat_params<double>(const BatchLat &L) { return L.pd; }

constexpr uint32_t kTileThreads = 256;  // threads per block of k_batch

struct Tile {
    int lat;
    uint32_t first;
};

struct GridBar {
    unsigned count;
    unsigned gen;
    int err;
    int skip;  // block that skips its first arrival (test hook), -1 for none
};

__device__ __forceinline__ uint64_t now_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier with a bounded wait: returns false (and raises bar->err)
// when the other blocks did not all arrive within timeout_ns.
__device__ bool grid_sync(GridBar *bar, unsigned nblocks, uint64_t timeout_ns, bool skip) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        volatile unsigned *vgen = &bar->gen;
        const unsigned g0 = *vgen;
        __threadfence();
        if (!skip && atomicAdd(&bar->count, 1u) == nblocks - 1) {
            atomicExch(&bar->count, 0u);
            __threadfence();
            atomicAdd(&bar->gen, 1u);
        }
        const uint64_t t0 = now_ns();
        while (*vgen == g0) {
            if (*(volatile int *)&bar->err || now_ns() - t0 > timeout_ns) {
                atomicExch(&bar->err, 1);
                ok = 0;
                break;
            }
            __nanosleep(200);
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// Minimum resident blocks per SM of the batched kernel (caps its registers;
// the cooperative grid is the resident-block count times the SM count).
#ifndef LBM_BATCH_MIN_BLOCKS
#define LBM_BATCH_MIN_BLOCKS 3
#endif

// Idx: type of the sparse population offsets, uint32_t unless a lattice of
// the launch has 19 units or more per 2^32 (as in the single-lattice kernels).
template <typename S, typename Idx>
__global__ void __launch_bounds__(256, sizeof(S) == 8 ? 1 : LBM_BATCH_MIN_BLOCKS) k_batch(const BatchLat *__restrict__ lats,
                                               const Tile *__restrict__ tiles,
                                               const int *__restrict__ ntiles_p,
                                               const int64_t *__restrict__ lat_steps, int nsteps,
                                               int nmeas,
                                               double *__restrict__ tile_part, int max_tiles,
                                               GridBar *bar, uint64_t timeout_ns) {
    using C = typename Store<S>::C;
    const int ntiles = *ntiles_p;
    __shared__ int skip_me;
    if (threadIdx.x == 0) skip_me = (*(volatile int *)&bar->skip == (int)blockIdx.x);
    __syncthreads();
    for (int s = 0; s < nsteps; ++s) {
        const int slot = s - (nsteps - nmeas);  // >= 0: one of the last nmeas steps
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
            const Tile tl = tiles[t];
            const BatchLat &L = lats[tl.lat];
            const Collide<C> &p = lat_params<C>(L);
            const bool odd = ((lat_steps[tl.lat] + s) & 1) != 0;
            S *A = (S *)L.pop;
            for (int r = 0; r < L.npt; ++r) {
                // sub-tile r: units first + 256 r .. first + 256 r + 255, the
                // same 256-unit group a single-lattice block covers
                const uint32_t u0 = tl.first + (uint32_t)r * blockDim.x;
                if (u0 >= L.units) break;  // block-uniform
                const uint32_t u = u0 + threadIdx.x;
                C jx = C(0), jy = C(0), jz = C(0);
                bool fl = false;
                if (u < L.units) {
                    // populations go through L2 only: other blocks wrote them
                    // in earlier steps of this launch (the index data is
                    // read-only)
                    if (L.layout == LBM_LAYOUT_SPARSE) {
                        fl = true;
                        if (odd)
                            aa_sparse_update<S, true, Idx, StoreL2<S>>(
                                A, L.sm, L.units, u, load_chk(L.sm.nb, u, L.units, L.sm.flag), p,
                                1.f, 1.f, jx, jy, jz);
                        else
                            aa_sparse_update<S, false, Idx, StoreL2<S>>(
                                A, L.sm, L.units, u, make_uint2(0u, 0u), p, 1.f, 1.f, jx, jy, jz);
                    } else {
                        const uint32_t w = L.lw[u];
                        fl = odd ? aa_dense_update<S, true, StoreL2<S>>(A, u, w, L.d, p, 1.f, 1.f,
                                                                        jx, jy, jz, L.sm.flag)
                                 : aa_dense_update<S, false, StoreL2<S>>(A, u, w, L.d, p, 1.f, 1.f,
                                                                         jx, jy, jz, L.sm.flag);
                    }
                }
                if (slot >= 0)  // the single-lattice block reduction
                    block_momentum_sum<C>(
                        jx, jy, jz, fl,
                        tile_part + ((size_t)slot * 2 * max_tiles + 2 * (size_t)t + r) * 3,
                        nullptr);
            }
        }
        if (s + 1 < nsteps && !grid_sync(bar, gridDim.x, timeout_ns, s == 0 && skip_me)) return;
    }
}

// U[i][slot][a] = (sum of lattice i's 256-unit partials) / N_i for the three
// measurement slots, in the order the single-lattice finalize uses: thread t
// adds partials t, t + 1024, ... in order, then a fixed shared-memory tree.
// Partial b of lattice i (units 256 b ..) sits in sub-tile b % npt of the
// lattice's tile b / npt.
__global__ void __launch_bounds__(1024) k_batch_finalize(const BatchLat *__restrict__ lats,
                                                         const int2 *__restrict__ lat_tiles,
                                                         const double *__restrict__ tile_part,
                                                         int max_tiles, double *U) {
    const int i = blockIdx.x;
    const int2 rng = lat_tiles[i];
    const int npt = lats[i].npt;
    const int nblk = rng.y > 0 ? (int)((lats[i].units + kTileThreads - 1) / kTileThreads) : 0;
    __shared__ double sm[3][1024];
    for (int slot = 0; slot < 3; ++slot) {
        const double *part = tile_part + (size_t)slot * 2 * max_tiles * 3;
        double acc[3] = {0.0, 0.0, 0.0};
        for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
            const size_t at = 2 * (size_t)(rng.x + b / npt) + b % npt;
#pragma unroll
            for (int a = 0; a < 3; ++a) acc[a] += part[3 * at + a];
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) sm[a][threadIdx.x] = acc[a];
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s)
#pragma unroll
                for (int a = 0; a < 3; ++a) sm[a][threadIdx.x] += sm[a][threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x < 3) U[(size_t)9 * i + 3 * slot + threadIdx.x] = sm[threadIdx.x][0] * lats[i].inv_N;
        __syncthreads();
    }
}

// ------------------------------------------------------ stepwise schedule
//
// Where the active lattices hold enough units to fill the GPU many times
// over, a grid barrier per step buys nothing over a kernel boundary, while
// the persistent kernel pays for its generality: populations through L2
// only, one unit per thread, both collision forms in one kernel and its
// register cap.  The stepwise schedule instead launches, per step, one
// kernel per class of lattices (layout x collision form x parity), each the
// multi-lattice twin of a single-lattice kernel: the two-node even step and
// the tiled odd step of the sparse layout, the dense AA step.  A block takes
// one tile of one lattice.  Per-node arithmetic and the per-256-unit group
// sums are those of the single-lattice kernels, and the partials of lattice i
// sit at part[slot][goff_i + group], summed in the single-lattice finalize's
// order, so members stay bitwise equal to lone runs.

#ifndef LBM_STEP_EVEN_NPT
#define LBM_STEP_EVEN_NPT 2
#endif
#ifndef LBM_STEP_ODD_MIN_BLOCKS
#define LBM_STEP_ODD_MIN_BLOCKS 3
#endif
constexpr uint32_t kEvenTile = 256 * LBM_STEP_EVEN_NPT;  // sparse even steps
constexpr uint32_t kOddTile = 1024;   // sparse odd steps: four units per thread
constexpr uint32_t kDenseTile = 256;  // dense AA steps: one unit per thread

struct StepRed {
    double *part;   // [nmeas][total groups][3], or nullptr on plain steps
    int slot;
    uint32_t ngroups;  // total groups (the slot stride)
};

__device__ __forceinline__ double *group_partial(const StepRed &r, const BatchLat &L, uint32_t g) {
    return r.part + 3 * ((size_t)r.slot * r.ngroups + L.goff + g);
}

template <typename S, int K, bool RED>
__global__ void __launch_bounds__(256, LBM_STEP_EVEN_NPT == 2 ? 2 : 3)
    k_step_sparse_even(const BatchLat *__restrict__ lats, const Tile *__restrict__ tiles, StepRed red) {
    using C = typename Store<S>::C;
    const Tile tl = tiles[blockIdx.x];
    const BatchLat &L = lats[tl.lat];
    // the lattice's collision parameters in shared memory: read where used,
    // instead of held in registers for the whole kernel
    __shared__ Collide<C> p;
    if (threadIdx.x == 0) p = lat_params<C>(L);
    __syncthreads();
    S *A = (S *)L.pop;
    const uint32_t Nf = L.units;
    const uint32_t k0 = tl.first + threadIdx.x, k1 = k0 + 256u;
    const bool v0 = k0 < Nf, v1 = LBM_STEP_EVEN_NPT == 2 && k1 < Nf;
    C g0[Q], g1[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) g0[j] = v0 ? Store<S>::ld(A + (uint32_t)j * Nf + k0, 1.f) : C(0);
#pragma unroll
    for (int j = 0; j < Q; ++j) g1[j] = v1 ? Store<S>::ld(A + (uint32_t)j * Nf + k1, 1.f) : C(0);
    C jx0 = C(0), jy0 = C(0), jz0 = C(0), jx1 = C(0), jy1 = C(0), jz1 = C(0);
    if (v0) {
        collide_as<K, C>(g0, p, jx0, jy0, jz0);
#pragma unroll
        for (int j = 0; j < Q; ++j) Store<S>::st(A + (uint32_t)j * Nf + k0, g0[opp(j)], 1.f);
    }
    if (v1) {
        collide_as<K, C>(g1, p, jx1, jy1, jz1);
#pragma unroll
        for (int j = 0; j < Q; ++j) Store<S>::st(A + (uint32_t)j * Nf + k1, g1[opp(j)], 1.f);
    }
    if (RED) {
        __shared__ double wsum[2][8][3];
        warp_momentum_store<C>(jx0, jy0, jz0, v0, wsum[0], L.sm.flag);
        warp_momentum_store<C>(jx1, jy1, jz1, v1, wsum[1], L.sm.flag);
        __syncthreads();
        const uint32_t g = tl.first / 256u;
        const int ng = LBM_STEP_EVEN_NPT == 2 && (g + 1u) * 256u < Nf ? 2 : 1;
        if ((int)threadIdx.x < 3 * ng) {
            const int r = threadIdx.x / 3, a = threadIdx.x % 3;
            group_partial(red, L, g + (uint32_t)r)[a] = group_momentum_total(wsum[r], a);
        }
    }
}

template <typename S, int K, bool RED>
__global__ void __launch_bounds__(256, LBM_STEP_ODD_MIN_BLOCKS)
    k_step_sparse_odd(const BatchLat *__restrict__ lats, const Tile *__restrict__ tiles, StepRed red) {
    using C = typename Store<S>::C;
    constexpr int NPT = (int)(kOddTile / 256);
    __shared__ double wsum[RED ? NPT : 1][8][3];
    const Tile tl = tiles[blockIdx.x];
    const BatchLat &L = lats[tl.lat];
    __shared__ Collide<C> p;
    if (threadIdx.x == 0) p = lat_params<C>(L);
    __syncthreads();
    S *A = (S *)L.pop;
    const SparseMap &m = L.sm;
    const uint32_t Nf = L.units;
    uint32_t k = tl.first + threadIdx.x;
    uint2 nxt = k < Nf ? __ldg(m.nb + k) : make_uint2(0u, 0u);
    const uint32_t g0 = tl.first / 256u;
    int groups = 0;
#pragma unroll 1
    for (int r = 0; r < NPT; ++r, k += 256u) {
        if ((g0 + (uint32_t)r) * 256u >= Nf) break;  // block-uniform
        const bool valid = k < Nf;
        const uint2 cur = nxt;
        if (r + 1 < NPT && k + 256u < Nf) nxt = __ldg(m.nb + k + 256u);
        C jx = C(0), jy = C(0), jz = C(0);
        if (valid)
            aa_sparse_update<S, true, uint32_t, Store<S>, K>(A, m, Nf, k, cur, p, 1.f, 1.f, jx, jy, jz);
        if (RED) warp_momentum_store<C>(jx, jy, jz, valid, wsum[RED ? r : 0], L.sm.flag);
        ++groups;
    }
    if (RED) {
        __syncthreads();
        if ((int)threadIdx.x < 3 * groups) {
            const int r = threadIdx.x / 3, a = threadIdx.x % 3;
            group_partial(red, L, g0 + (uint32_t)r)[a] = group_momentum_total(wsum[r], a);
        }
    }
}

template <typename S, bool ODD, int K, bool RED>
__global__ void __launch_bounds__(256)
    k_step_dense(const BatchLat *__restrict__ lats, const Tile *__restrict__ tiles, StepRed red) {
    using C = typename Store<S>::C;
    const Tile tl = tiles[blockIdx.x];
    const BatchLat &L = lats[tl.lat];
    __shared__ Collide<C> p;
    if (threadIdx.x == 0) p = lat_params<C>(L);
    __syncthreads();
    const uint32_t n = tl.first + threadIdx.x;
    const uint32_t w = n < L.units ? L.lw[n] : SOLID_BIT;
    C jx = C(0), jy = C(0), jz = C(0);
    const bool fluid = aa_dense_update<S, ODD, Store<S>, K>((S *)L.pop, n, w, L.d, p, 1.f, 1.f, jx,
                                                            jy, jz, L.sm.flag);
    if (RED) block_momentum_sum<C>(jx, jy, jz, fluid, group_partial(red, L, tl.first / 256u),
                                   L.sm.flag);
}

// U[i][slot][a] for the lattices flagged in `want`: the sum of lattice i's
// group partials of each measured slot over N_i, in the single-lattice
// finalize's order (thread t adds groups t, t + 1024, ..., then a fixed
// shared-memory tree).
__global__ void __launch_bounds__(1024) k_step_finalize(const BatchLat *__restrict__ lats,
                                                        const char *__restrict__ want,
                                                        const double *__restrict__ part,
                                                        uint32_t ngroups, int nmeas, double *U) {
    const int i = blockIdx.x;
    if (!want[i]) return;
    const uint32_t ng = (lats[i].units + 255u) / 256u;
    __shared__ double sm[3][1024];
    for (int slot = 0; slot < nmeas; ++slot) {
        const double *pp = part + 3 * ((size_t)slot * ngroups + lats[i].goff);
        double acc[3] = {0.0, 0.0, 0.0};
        for (uint32_t b = threadIdx.x; b < ng; b += blockDim.x)
#pragma unroll
            for (int a = 0; a < 3; ++a) acc[a] += pp[3 * (size_t)b + a];
#pragma unroll
        for (int a = 0; a < 3; ++a) sm[a][threadIdx.x] = acc[a];
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s)
#pragma unroll
                for (int a = 0; a < 3; ++a) sm[a][threadIdx.x] += sm[a][threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x < 3) U[(size_t)9 * i + 3 * slot + threadIdx.x] = sm[threadIdx.x][0] * lats[i].inv_N;
        __syncthreads();
    }
}

}  // namespace lbm

using namespace lbm;

// One class of the stepwise schedule: lattices of one layout and collision
// form whose step count had parity `parity` at the chunk's start.  Sparse
// classes keep an even-step and an odd-step tile list, dense classes one.
struct StepClass {
    int layout, trt;
    int rep;               // a member lattice: its step count gives the class's parity
    int even_off, even_n;  // tiles in d_step_tiles
    int odd_off, odd_n;
};

struct lbm_batch {
    int n;
    std::vector<lbm_ctx *> ctx;
    lbm_batch_options opt;
    cudaStream_t stream;
    bool own_stream;
    std::vector<int> layout, npt;
    std::vector<char> solo;  // run alone with the single-lattice kernels
    std::vector<char> active;
    std::vector<int64_t> steps;
    std::vector<int> status;
    std::vector<double> Ua, Ub;
    BatchLat *d_lats;
    Tile *d_tiles;
    int *d_ntiles;
    int2 *d_lat_tiles;
    int64_t *d_steps, *h_steps;
    double *d_tile_part;
    int max_tiles;
    GridBar *d_bar;
    double *d_U, *h_U;
    int *h_err;
    int grid;
    cudaGraphExec_t gexec;
    bool graph_ok;
    bool failed;
    int64_t launches;
    uint64_t timeout_ns;
    // stepwise schedule
    std::vector<StepClass> classes;
    std::vector<int> group_end;  // classes of group g: [group_end[g-1], group_end[g])
    std::vector<int> direct;     // active lattices stepped with their own kernels
    std::vector<char> in_direct;  // automatic schedule: left out of the persistent launch
    Tile *d_step_tiles;
    int max_step_tiles;
    double *d_step_part;
    uint32_t ngroups;
    char *d_want;
    int64_t stepwise_chunks, persistent_chunks;
    std::vector<uint32_t> goff;
    // automatic schedule: side streams for lattices stepped concurrently
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> side_done;
    cudaEvent_t fork;
    bool side_tried;  // side streams created (or their creation failed) once
    bool wide;        // a lattice needs 64-bit offsets: the persistent kernel takes them
};

extern "C" {

void lbm_batch_default_options(lbm_batch_options *o) {
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->precision = LBM_FP32_SHIFTED;
    o->layout = -1;
    o->nodes_per_thread = 0;
    o->check_interval = 100;
    o->max_steps = 1000000;
    o->use_graph = 1;
    o->barrier_timeout_ms = 2000;
    o->test_skip_block = -1;
    o->stop_rule = 0;
    o->solo = 1;
    o->schedule = 0;
}

void lbm_batch_destroy(lbm_batch *b) {
    if (!b) return;
    for (cudaStream_t st : b->side) cudaStreamSynchronize(st);
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (cudaStream_t st : b->side) cudaStreamDestroy(st);
    for (cudaEvent_t ev : b->side_done) cudaEventDestroy(ev);
    if (b->fork) cudaEventDestroy(b->fork);
    for (lbm_ctx *c : b->ctx) lbm_destroy(c);
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    cudaFree(b->d_lats);
    cudaFree(b->d_tiles);
    cudaFree(b->d_ntiles);
    cudaFree(b->d_lat_tiles);
    cudaFree(b->d_steps);
    cudaFree(b->d_tile_part);
    cudaFree(b->d_bar);
    cudaFree(b->d_U);
    cudaFree(b->d_step_tiles);
    cudaFree(b->d_step_part);
    cudaFree(b->d_want);
    cudaFreeHost(b->h_steps);
    cudaFreeHost(b->h_U);
    cudaFreeHost(b->h_err);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

}  // extern "C"

namespace {

BatchLat make_lat(const lbm_ctx *c, int npt) {
    BatchLat L;
    memset(&L, 0, sizeof L);
    L.layout = c->opt.layout;
    L.npt = npt;
    L.units = (uint32_t)(c->opt.layout == LBM_LAYOUT_SPARSE ? c->Nf : c->N);
    L.pop = c->d_pop[0];
    L.lw = c->d_lw;
    if (c->opt.layout == LBM_LAYOUT_SPARSE) L.sm = sparse_map(c);
    L.sm.flag = c->d_flag;  // the member's own flag (bounds-check build)
    L.d = Dims{c->Lx, c->Ly, c->Lz, (uint32_t)c->N};
    L.pf = make_collide<float>(c->s, c->F, c->opt.linear_eq, c->opt.collision == 0);
    L.pd = make_collide<double>(c->s, c->F, c->opt.linear_eq, c->opt.collision == 0);
    L.inv_N = 1.0 / (double)c->N;
    return L;
}

int ntiles_of(const BatchLat &L) { return (int)((L.units + kTileThreads * L.npt - 1) / (kTileThreads * L.npt)); }

// The persistent kernel for a precision and offset width.
const void *batch_kernel(int precision, bool wide) {
    if (precision == LBM_FP64)
        return wide ? (const void *)k_batch<double, size_t> : (const void *)k_batch<double, uint32_t>;
    return wide ? (const void *)k_batch<float, size_t> : (const void *)k_batch<float, uint32_t>;
}

// Whether lattice L needs 64-bit population offsets.
bool wide_lat(const BatchLat &L) { return 19 * (uint64_t)L.units >= (uint64_t(1) << 32); }

// Cooperative grid: every block resident, for either offset width.
int coop_grid(int precision) {
    int dev = 0, sms = 0, per = 1 << 30;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    for (const bool wide : {false, true}) {
        int p = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p, batch_kernel(precision, wide), 256, 0) !=
            cudaSuccess) {
            p = 0;
            cudaGetLastError();
        }
        per = p < per ? p : per;
    }
    return sms * (per > 0 ? per : 1);
}

// ---- stepwise schedule (host side)

uint32_t groups_of(const BatchLat &L) { return (L.units + 255u) / 256u; }
bool lat_trt(const lbm_batch *b, const BatchLat &L) {
    return b->opt.precision == LBM_FP64 ? L.pd.trt != 0 : L.pf.trt != 0;
}

// Tiles of lattice i for the stepwise kernels: sparse lattices an even-step
// list (kEvenTile units per tile) and an odd-step list (kOddTile), dense
// lattices one list (kDenseTile).
void step_tiles_of(const BatchLat &L, int i, std::vector<Tile> &even, std::vector<Tile> &odd) {
    if (L.layout == LBM_LAYOUT_SPARSE) {
        for (uint32_t u = 0; u < L.units; u += kEvenTile) even.push_back(Tile{i, u});
        for (uint32_t u = 0; u < L.units; u += kOddTile) odd.push_back(Tile{i, u});
    } else {
        for (uint32_t u = 0; u < L.units; u += kDenseTile) even.push_back(Tile{i, u});
    }
}

// Launches one stepwise kernel over `n` tiles of one class at parity par.
cudaError_t launch_step_kernel(cudaStream_t st, const BatchLat *d_lats, const Tile *tiles, int n,
                               int layout, bool trt, int par, const StepRed &red) {
    if (n <= 0) return cudaSuccess;
    const bool R = red.part != nullptr;
#define LBM_STEP_LAUNCH(KERNEL, ...)                                                             \
    do {                                                                                         \
        if (trt) {                                                                               \
            if (R) KERNEL<__VA_ARGS__, kCollideTrt, true><<<n, 256, 0, st>>>(d_lats, tiles, red); \
            else KERNEL<__VA_ARGS__, kCollideTrt, false><<<n, 256, 0, st>>>(d_lats, tiles, red);  \
        } else {                                                                                 \
            if (R) KERNEL<__VA_ARGS__, kCollideMrt, true><<<n, 256, 0, st>>>(d_lats, tiles, red); \
            else KERNEL<__VA_ARGS__, kCollideMrt, false><<<n, 256, 0, st>>>(d_lats, tiles, red);  \
        }                                                                                        \
    } while (0)
    if (layout == LBM_LAYOUT_SPARSE) {
        if (par == 0) LBM_STEP_LAUNCH(k_step_sparse_even, float);
        else LBM_STEP_LAUNCH(k_step_sparse_odd, float);
    } else {
        if (par == 0) LBM_STEP_LAUNCH(k_step_dense, float, false);
        else LBM_STEP_LAUNCH(k_step_dense, float, true);
    }
#undef LBM_STEP_LAUNCH
    return cudaGetLastError();
}

// Bytes a lattice's steps touch: its populations and, per unit, the index
// record or link word.
size_t lat_bytes(const lbm_batch *b, const BatchLat &L) {
    const size_t elem = b->opt.precision == LBM_FP64 ? 8 : 4;
    return (size_t)L.units * (Q * elem + (L.layout == LBM_LAYOUT_SPARSE ? 8 : 4));
}

// A lattice with at least this many units fills the GPU by itself: it runs
// each chunk with its own single-lattice kernels (whose parameters sit in
// the constant bank; at 96^3 they stepped 40% faster than the multi-lattice
// kernels with one lattice per launch), on the batch's stream, its chunk
// replayed from its own CUDA graph, its state staying in L2 from step to
// step where it fits.
#ifndef LBM_STEP_DIRECT_UNITS
#define LBM_STEP_DIRECT_UNITS 100000
#endif
constexpr int64_t kDirectUnits = LBM_STEP_DIRECT_UNITS;

// Under the automatic schedule, up to LBM_BATCH_STREAMS such lattices run
// their chunks at the same time, each on a side stream, as long as their
// states together fit LBM_BATCH_CONC_L2_PERCENT of the L2 cache.  A lone
// single-lattice launch leaves most SMs idle in its last wave, and between
// its kernels; concurrent lattices fill those gaps.  Groups run in turn,
// forked from and joined back into the batch's stream.
#ifndef LBM_BATCH_STREAMS
#define LBM_BATCH_STREAMS 4
#endif
#ifndef LBM_BATCH_CONC_L2_PERCENT
#define LBM_BATCH_CONC_L2_PERCENT 60
#endif

// Creates the side streams and events once; returns how many are usable
// (0: every lattice runs on the batch's stream).
// A failed creation is not retried; its error is cleared (and only then).
static int side_streams(lbm_batch *b) {
    if (b->side_tried || LBM_BATCH_STREAMS < 2) return (int)b->side.size();
    b->side_tried = true;
    if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) {
        b->fork = nullptr;
        cudaGetLastError();
        return 0;
    }
    for (int j = 0; j < LBM_BATCH_STREAMS; ++j) {
        cudaStream_t st = nullptr;
        cudaEvent_t ev = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            break;
        }
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            cudaStreamDestroy(st);
            break;
        }
        b->side.push_back(st);
        b->side_done.push_back(ev);
    }
    return (int)b->side.size();
}

// Enqueues one chunk (plain steps, then nmeas measuring steps) of each
// lattice in `ids` with its own kernels: in groups of up to
// LBM_BATCH_STREAMS lattices on the side streams, each group joined into
// the batch's stream before the next one forks.  Groups are packed first
// fit, largest state first, so that a large lattice shares its group with
// small ones where the budget allows.  The lattices' results are bitwise
// those of a sequential run: no lattice reads another's data.
static int run_direct(lbm_batch *b, const std::vector<int> &ids, const std::vector<BatchLat> &lats,
                      int64_t plain, int nmeas) {
    const int ns = side_streams(b);
    int dev = 0, l2 = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
    const size_t budget = (size_t)(l2 > 0 ? l2 : (64 << 20)) * LBM_BATCH_CONC_L2_PERCENT / 100;
    std::vector<int> order(ids);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        return lat_bytes(b, lats[x]) > lat_bytes(b, lats[y]);
    });
    std::vector<std::vector<int>> groups;
    std::vector<size_t> used;
    for (const int i : order) {
        const size_t by = lat_bytes(b, lats[i]);
        size_t g = 0;
        while (g < groups.size() && !((int)groups[g].size() < ns && used[g] + by <= budget)) ++g;
        if (g == groups.size()) {
            groups.emplace_back();
            used.push_back(0);
        }
        groups[g].push_back(i);
        used[g] += by;
    }
    for (const std::vector<int> &grp : groups) {
        const bool fork = grp.size() > 1;
        if (fork && cudaEventRecord(b->fork, b->stream) != cudaSuccess) return LBM_ECUDA;
        for (size_t m = 0; m < grp.size(); ++m) {
            lbm_ctx *c = b->ctx[grp[m]];
            const cudaStream_t own = c->stream;
            const int j = (int)m;
            if (fork) {
                if (cudaStreamWaitEvent(b->side[j], b->fork, 0) != cudaSuccess) return LBM_ECUDA;
                c->stream = b->side[j];
            }
            const int64_t l0 = c->launches;
            const int rc = enqueue_measured_chunk(c, plain, nmeas);
            c->stream = own;
            b->launches += c->launches - l0;
            if (rc != LBM_OK) return rc;
            if (fork && (cudaEventRecord(b->side_done[j], b->side[j]) != cudaSuccess ||
                         cudaStreamWaitEvent(b->stream, b->side_done[j], 0) != cudaSuccess))
                return LBM_ECUDA;
        }
    }
    return LBM_OK;
}

// Share of the L2 cache a group of lattices may fill (percent).
#ifndef LBM_STEP_L2_PERCENT
#define LBM_STEP_L2_PERCENT 60
#endif

// Rebuilds the groups, classes and tile lists of the active lattices.  The
// active lattices are packed, in order, into groups whose states together
// fit LBM_STEP_L2_PERCENT of the L2 cache (a larger lattice is a group of
// its own); a chunk runs each group through all its steps before the next,
// so a group's populations stay in L2 from one step to the next.
cudaError_t upload_step_tiles(lbm_batch *b, const std::vector<BatchLat> &lats) {
    int dev = 0, l2 = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
    const size_t budget = (size_t)(l2 > 0 ? l2 : (64 << 20)) * LBM_STEP_L2_PERCENT / 100;
    std::vector<char> want(b->n, 0);
    std::vector<Tile> all;
    b->classes.clear();
    b->group_end.clear();
    size_t used = 0;
    std::map<int, std::pair<std::vector<Tile>, std::vector<Tile>>> lists;
    std::map<int, int> rep;
    auto flush = [&]() {
        for (auto &kv : lists) {
            StepClass c;
            c.layout = kv.first / 4;
            c.trt = (kv.first >> 1) & 1;
            c.rep = rep[kv.first];
            c.even_off = (int)all.size();
            c.even_n = (int)kv.second.first.size();
            all.insert(all.end(), kv.second.first.begin(), kv.second.first.end());
            c.odd_off = (int)all.size();
            c.odd_n = (int)kv.second.second.size();
            all.insert(all.end(), kv.second.second.begin(), kv.second.second.end());
            b->classes.push_back(c);
        }
        if (!lists.empty()) b->group_end.push_back((int)b->classes.size());
        lists.clear();
        rep.clear();
        used = 0;
    };
    b->direct.clear();
    for (int i = 0; i < b->n; ++i) {
        if (!b->active[i]) continue;
        if ((int64_t)lats[i].units >= kDirectUnits) {  // fills the GPU by itself
            b->direct.push_back(i);
            continue;
        }
        want[i] = 1;
        const size_t bytes = lat_bytes(b, lats[i]);
        if (used > 0 && used + bytes > budget) flush();
        used += bytes;
        const int key = lats[i].layout * 4 + (lat_trt(b, lats[i]) ? 2 : 0) + (int)(b->ctx[i]->steps & 1);
        auto &l = lists[key];
        step_tiles_of(lats[i], i, l.first, l.second);
        rep.emplace(key, i);
    }
    flush();
    cudaError_t e = cudaSuccess;
    if (!all.empty())
        e = cudaMemcpyAsync(b->d_step_tiles, all.data(), sizeof(Tile) * all.size(),
                            cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_want, want.data(), (size_t)b->n, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);  // host vectors go out of scope
    return e;
}

// One chunk of K steps under the stepwise schedule: per step one launch per
// class, the last nmeas steps measuring; then the per-lattice sums and the
// copy of the results.
cudaError_t enqueue_step_chunk(lbm_batch *b) {
    const int K = b->opt.check_interval;
    const int nmeas = b->opt.stop_rule == 1 ? 3 : 2;
    for (const int i : b->direct) {  // lattices that fill the GPU alone
        lbm_ctx *c = b->ctx[i];
        const int64_t l0 = c->launches;
        const int rc = enqueue_measured_chunk(c, K - nmeas, nmeas);
        if (rc != LBM_OK) return cudaErrorUnknown;
        b->launches += c->launches - l0;
    }
    int c0 = 0;
    for (const int c1 : b->group_end) {  // the groups one after another
        for (int s = 0; s < K; ++s) {
            const int slot = s - (K - nmeas);
            StepRed red{slot >= 0 ? b->d_step_part : nullptr, slot, b->ngroups};
            for (int ci = c0; ci < c1; ++ci) {
                const StepClass &c = b->classes[ci];
                const int par = (int)((b->ctx[c.rep]->steps + s) & 1);
                const bool odd_list = c.layout == LBM_LAYOUT_SPARSE && par == 1;
                cudaError_t e = launch_step_kernel(
                    b->stream, b->d_lats, b->d_step_tiles + (odd_list ? c.odd_off : c.even_off),
                    odd_list ? c.odd_n : c.even_n, c.layout, c.trt != 0, par, red);
                if (e != cudaSuccess) return e;
                b->launches++;
            }
        }
        c0 = c1;
    }
    k_step_finalize<<<b->n, 1024, 0, b->stream>>>(b->d_lats, b->d_want, b->d_step_part, b->ngroups,
                                                  nmeas, b->d_U);
    b->launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    *b->h_err = 0;
    e = cudaMemcpyAsync(b->h_U, b->d_U, sizeof(double) * 9 * b->n, cudaMemcpyDeviceToHost,
                        b->stream);
    for (const int i : b->direct)  // their measured slots, after the bulk copy
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->h_U + 9 * (size_t)i, b->ctx[i]->d_U, sizeof(double) * 3 * nmeas,
                                cudaMemcpyDeviceToHost, b->stream);
    return e;
}

// Active lattices hold at least this many units: run the chunk stepwise
// (four waves of the persistent kernel's resident threads).
int64_t stepwise_min_units(const lbm_batch *b) { return 4 * (int64_t)b->grid * kTileThreads; }

// Autotuner for the stepwise schedule: device time of `steps` steps of the
// stepwise kernels over enough copies of lattice c's tiles to fill the GPU
// (about four waves), per copy.  The copies update the same populations, so
// the scratch context's values are meaningless afterwards; only the time
// is used.
float time_candidate_step(lbm_batch *b, lbm_ctx *c, int steps) {
    BatchLat L = make_lat(c, 1);
    L.goff = 0;
    // copies up to four waves of threads, within one group's share of L2
    int dev = 0, l2 = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
    const int64_t budget = (int64_t)(l2 > 0 ? l2 : (64 << 20)) * LBM_STEP_L2_PERCENT / 100;
    const int64_t target = stepwise_min_units(b);
    const int64_t units = L.units ? L.units : 1;
    int64_t R = (target + units - 1) / units;
    const int64_t fit = budget / (int64_t)(lat_bytes(b, L) ? lat_bytes(b, L) : 1);
    if (R > fit) R = fit;
    if (R < 1) R = 1;
    std::vector<Tile> even, odd;
    for (int r = 0; r < R; ++r) step_tiles_of(L, 0, even, odd);
    BatchLat *d_l = nullptr;
    Tile *d_t = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float ms = INFINITY;
    const size_t nt = even.size() + odd.size();
    if (cudaMalloc(&d_l, sizeof L) == cudaSuccess && cudaMalloc(&d_t, sizeof(Tile) * nt) == cudaSuccess &&
        cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
        cudaMemcpyAsync(d_l, &L, sizeof L, cudaMemcpyHostToDevice, b->stream);
        cudaMemcpyAsync(d_t, even.data(), sizeof(Tile) * even.size(), cudaMemcpyHostToDevice, b->stream);
        if (!odd.empty())
            cudaMemcpyAsync(d_t + even.size(), odd.data(), sizeof(Tile) * odd.size(),
                            cudaMemcpyHostToDevice, b->stream);
        const StepRed none{nullptr, 0, 0};
        const bool trt = lat_trt(b, L);
        cudaError_t e = cudaSuccess;
        cudaEventRecord(e0, b->stream);
        for (int s = 0; s < steps && e == cudaSuccess; ++s) {
            const int par = s & 1;
            const bool ol = L.layout == LBM_LAYOUT_SPARSE && par == 1;
            e = launch_step_kernel(b->stream, d_l, ol ? d_t + even.size() : d_t,
                                   (int)(ol ? odd.size() : even.size()), L.layout, trt, par, none);
            b->launches++;
        }
        cudaEventRecord(e1, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (e == cudaSuccess) {
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= (float)R;  // per copy
        }
        cudaGetLastError();
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(d_l);
    cudaFree(d_t);
    return ms;
}

// Uploads the tile table of the active lattices.
cudaError_t upload_tiles(lbm_batch *b, const std::vector<BatchLat> &lats) {
    std::vector<Tile> tiles;
    std::vector<int2> ranges(b->n, make_int2(0, 0));
    for (int i = 0; i < b->n; ++i) {
        if (!b->active[i] || (i < (int)b->in_direct.size() && b->in_direct[i])) continue;
        const int nt = ntiles_of(lats[i]);
        ranges[i] = make_int2((int)tiles.size(), nt);
        for (int t = 0; t < nt; ++t) tiles.push_back(Tile{i, (uint32_t)t * kTileThreads * lats[i].npt});
    }
    const int nt = (int)tiles.size();
    cudaError_t e = cudaSuccess;
    if (nt) e = cudaMemcpyAsync(b->d_tiles, tiles.data(), sizeof(Tile) * nt, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_ntiles, &nt, sizeof(int), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_lat_tiles, ranges.data(), sizeof(int2) * b->n, cudaMemcpyHostToDevice,
                            b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);  // host vectors go out of scope
    return e;
}

cudaError_t enqueue_chunk(lbm_batch *b) {
    cudaError_t e = cudaMemcpyAsync(b->d_steps, b->h_steps, sizeof(int64_t) * b->n,
                                    cudaMemcpyHostToDevice, b->stream);
    if (e != cudaSuccess) return e;
    int K = b->opt.check_interval;
    int nmeas = b->opt.stop_rule == 1 ? 3 : 2;
    void *args[] = {&b->d_lats, &b->d_tiles, &b->d_ntiles, &b->d_steps, &K, &nmeas,
                    &b->d_tile_part, &b->max_tiles, &b->d_bar, &b->timeout_ns};
    const void *fn = batch_kernel(b->opt.precision, b->wide);
    e = cudaLaunchCooperativeKernel(fn, dim3(b->grid), dim3(kTileThreads), args, 0, b->stream);
    if (e != cudaSuccess) return e;
    k_batch_finalize<<<b->n, 1024, 0, b->stream>>>(b->d_lats, b->d_lat_tiles, b->d_tile_part,
                                                  b->max_tiles, b->d_U);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(b->h_U, b->d_U, sizeof(double) * 9 * b->n, cudaMemcpyDeviceToHost, b->stream);
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(b->h_err, &b->d_bar->err, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
}

// Autotuner: device time of `steps` batch steps of one lattice in a given
// layout and nodes-per-thread, measured with events on the batch stream.
float time_candidate(lbm_batch *b, lbm_ctx *c, int npt, int steps) {
    BatchLat L = make_lat(c, npt);
    const int nt = ntiles_of(L);
    std::vector<Tile> tiles;
    for (int t = 0; t < nt; ++t) tiles.push_back(Tile{0, (uint32_t)t * kTileThreads * npt});
    BatchLat *d_l = nullptr;
    Tile *d_t = nullptr;
    int *d_n = nullptr;
    int64_t *d_s = nullptr;
    double *d_p = nullptr;
    GridBar *d_b = nullptr;
    float ms = INFINITY;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaMalloc(&d_l, sizeof L) == cudaSuccess && cudaMalloc(&d_t, sizeof(Tile) * nt) == cudaSuccess &&
        cudaMalloc(&d_n, sizeof(int)) == cudaSuccess && cudaMalloc(&d_s, sizeof(int64_t)) == cudaSuccess &&
        cudaMalloc(&d_p, sizeof(double) * 18 * nt) == cudaSuccess &&
        cudaMalloc(&d_b, sizeof(GridBar)) == cudaSuccess && cudaEventCreate(&e0) == cudaSuccess &&
        cudaEventCreate(&e1) == cudaSuccess) {
        const int64_t zero = 0;
        GridBar gb{0u, 0u, 0, -1};
        cudaMemcpyAsync(d_l, &L, sizeof L, cudaMemcpyHostToDevice, b->stream);
        cudaMemcpyAsync(d_t, tiles.data(), sizeof(Tile) * nt, cudaMemcpyHostToDevice, b->stream);
        cudaMemcpyAsync(d_n, &nt, sizeof(int), cudaMemcpyHostToDevice, b->stream);
        cudaMemcpyAsync(d_s, &zero, sizeof zero, cudaMemcpyHostToDevice, b->stream);
        cudaMemcpyAsync(d_b, &gb, sizeof gb, cudaMemcpyHostToDevice, b->stream);
        int grid = b->grid < nt ? b->grid : nt;
        int maxt = nt;
        int nmeas = 2;
        void *args[] = {&d_l, &d_t, &d_n, &d_s, &steps, &nmeas, &d_p, &maxt, &d_b, &b->timeout_ns};
        const void *fn = batch_kernel(b->opt.precision, wide_lat(L));
        cudaEventRecord(e0, b->stream);
        cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kTileThreads), args, 0, b->stream);
        cudaEventRecord(e1, b->stream);
        int err = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&err, &d_b->err, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (e == cudaSuccess && !err) cudaEventElapsedTime(&ms, e0, e1);
        b->launches++;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(d_l);
    cudaFree(d_t);
    cudaFree(d_n);
    cudaFree(d_s);
    cudaFree(d_p);
    cudaFree(d_b);
    return ms;
}

// Smallest lattice (units) offered to run alone: four waves of the batched
// kernel's resident threads.
int64_t solo_min_units() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return 4 * (int64_t)sms * LBM_BATCH_MIN_BLOCKS * kTileThreads;
}

// Device time of `steps` single-lattice steps of context c on the batch's
// stream (launch gaps included): the cost of running the lattice alone.
float time_solo(lbm_batch *b, lbm_ctx *c, int steps) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float ms = INFINITY;
    if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
        cudaEventRecord(e0, c->stream);
        for (int t = 0; t < steps; ++t) launch_step(c, false);
        cudaEventRecord(e1, c->stream);
        if (cudaStreamSynchronize(c->stream) == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    (void)b;
    return ms;
}

std::string mask_key(const lbm_lattice_desc &d) {
    const size_t N = (size_t)d.dims[0] * d.dims[1] * d.dims[2];
    uint64_t h = 1469598103934665603ull;  // FNV-1a over the mask bytes
    for (size_t i = 0; i < N; ++i) h = (h ^ d.mask[i]) * 1099511628211ull;
    char buf[96];
    snprintf(buf, sizeof buf, "%d.%d.%d.%016llx", d.dims[0], d.dims[1], d.dims[2],
             (unsigned long long)h);
    return buf;
}

}  // namespace

extern "C" {

int lbm_batch_create(lbm_batch **out, int32_t n, const lbm_lattice_desc *desc,
                     const lbm_batch_options *opt) {
    if (!out || n <= 0 || !desc) return LBM_EINVAL;
    *out = nullptr;
    lbm_batch_options o;
    lbm_batch_default_options(&o);
    if (opt) o = *opt;
    if (o.precision != LBM_FP32_SHIFTED && o.precision != LBM_FP64) return LBM_EINVAL;
    if (o.layout != -1 && o.layout != LBM_LAYOUT_AA && o.layout != LBM_LAYOUT_SPARSE) return LBM_EINVAL;
    if (o.nodes_per_thread < 0 || o.nodes_per_thread > 2) return LBM_EINVAL;
    if (o.check_interval < 2) o.check_interval = 2;
    if (o.max_steps <= 0) o.max_steps = 1000000;
    if (o.barrier_timeout_ms <= 0) o.barrier_timeout_ms = 2000;
    if (o.stop_rule != 0 && o.stop_rule != 1) return LBM_EINVAL;
    if (o.stop_rule == 1 && o.check_interval < 3) o.check_interval = 3;
    if (o.solo < 0 || o.solo > 2) return LBM_EINVAL;
    if (o.schedule < 0 || o.schedule > 2) return LBM_EINVAL;
    if (o.schedule == 2 && o.precision != LBM_FP32_SHIFTED) return LBM_EINVAL;
    lbm_batch *b = new (std::nothrow) lbm_batch();
    if (!b) return LBM_ENOMEM;
    b->n = n;
    b->opt = o;
    b->timeout_ns = (uint64_t)o.barrier_timeout_ms * 1000000ull;
    auto fail = [&](int rc) {
        lbm_batch_destroy(b);
        return rc;
    };
    cudaError_t e;
    if (o.cuda_stream) {
        b->stream = (cudaStream_t)o.cuda_stream;
    } else {
        e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return fail(launch_error(e));
        b->own_stream = true;
    }
    b->grid = coop_grid(o.precision);
    lbm_options lo;
    lbm_default_options(&lo);
    lo.precision = o.precision;
    lo.check_interval = o.check_interval;
    lo.linear_eq = o.linear_eq;
    lo.max_steps = o.max_steps;
    lo.cuda_stream = b->stream;
    // Lattices that share the persistent launch move their whole state every
    // step.  When those states together exceed the L2 share, the layout of
    // such a lattice is the one with fewer bytes per step (dense: 19 values
    // and a link word per voxel; sparse: 19 values and an 8-byte record per
    // fluid node), not the faster one when timed alone: alone, a small
    // lattice stays in L2 and its time is the grid barriers', which favours
    // the dense layout's simpler indexing.  (The 378-lattice subset sweep:
    // timed choices, mostly dense, 0.555 s; every lattice sparse 0.477 s.)
    std::vector<std::string> keys(n);
    std::map<std::string, std::pair<int64_t, int64_t>> counts;  // image -> (N, N_f)
    for (int i = 0; i < n; ++i) {
        const lbm_lattice_desc &d = desc[i];
        if (!d.mask || d.dims[0] <= 0 || d.dims[1] <= 0 || d.dims[2] <= 0) return fail(LBM_EINVAL);
        // the size lbm_create accepts, checked before any mask byte is read
        const int64_t n01 = (int64_t)d.dims[0] * d.dims[1];
        if (n01 >= (int64_t(1) << 31) || n01 * d.dims[2] >= (int64_t(1) << 31)) return fail(LBM_EINVAL);
        keys[i] = mask_key(d);
        if (counts.count(keys[i])) continue;
        const int64_t N = (int64_t)d.dims[0] * d.dims[1] * d.dims[2];
        int64_t nf = 0;
        for (int64_t v = 0; v < N; ++v) nf += d.mask[v] == 0;
        counts[keys[i]] = std::make_pair(N, nf);
    }
    const int64_t val_bytes = 19 * (o.precision == LBM_FP64 ? 8 : 4);
    auto dense_bytes = [&](const std::pair<int64_t, int64_t> &c) { return c.first * (val_bytes + 4); };
    auto sparse_bytes = [&](const std::pair<int64_t, int64_t> &c) { return c.second * (val_bytes + 8); };
    auto shares_launch = [&](const std::pair<int64_t, int64_t> &c) {
        return o.schedule == 1 || c.second < kDirectUnits;
    };
    bool by_bytes = false;
    if (o.layout == -1 && o.schedule != 2) {
        int dev = 0, l2 = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
        double shared = 0.0;
        for (int i = 0; i < n; ++i) {
            const auto &c = counts[keys[i]];
            if (shares_launch(c)) shared += (double)std::min(dense_bytes(c), sparse_bytes(c));
        }
        by_bytes = shared > (double)(l2 > 0 ? l2 : (64 << 20)) * LBM_STEP_L2_PERCENT / 100.0;
    }
    // autotune per distinct image: layout and nodes per thread
    std::map<std::string, std::pair<int, int>> tuned;
    b->layout.resize(n);
    b->npt.resize(n);
    for (int i = 0; i < n; ++i) {
        const lbm_lattice_desc &d = desc[i];
        int lay = o.layout, np = o.nodes_per_thread;
        if (lay == -1 || np == 0) {
            const std::string &key = keys[i];
            const auto &cnt = counts[key];
            // by bytes: the one layout this image is offered (-1: both)
            const int pick = by_bytes && shares_launch(cnt)
                                 ? (sparse_bytes(cnt) <= dense_bytes(cnt) ? LBM_LAYOUT_SPARSE
                                                                          : LBM_LAYOUT_AA)
                                 : -1;
            auto it = tuned.find(key);
            if (it == tuned.end()) {
                // Each candidate layout is timed as it will run: under the
                // automatic schedule, alone with its own kernels where it
                // fills the GPU, else in the persistent kernel; under the
                // grouped stepwise schedule, on the stepwise kernels (copies
                // of the lattice filling the GPU).  Units per thread are
                // timed on the persistent kernel.
                const bool stepwise = o.schedule != 1;
                float best = INFINITY, best_step = INFINITY;
                int bl = LBM_LAYOUT_AA, bn = 1;
                int bn_of[3] = {1, 1, 1};
                for (int cl : {LBM_LAYOUT_AA, LBM_LAYOUT_SPARSE}) {
                    if (lay != -1 && cl != lay) continue;
                    if (pick != -1 && cl != pick) continue;
                    lbm_options to = lo;
                    to.layout = cl;
                    lbm_ctx *c = nullptr;
                    int rc = d.set >= 0 ? lbm_create(&c, d.mask, d.dims, d.set, d.tau, d.Lambda, d.force, &to)
                                        : lbm_create_rates(&c, d.mask, d.dims, d.s, d.force, &to);
                    if (rc != LBM_OK) return fail(rc);
                    const int64_t un = cl == LBM_LAYOUT_SPARSE ? c->Nf : c->N;
                    const bool alone = un >= kDirectUnits;
                    float best_here = INFINITY;
                    for (int cn : {1, 2}) {
                        if (np != 0 && cn != np) continue;
                        if (o.solo == 2) continue;
                        // layout by bytes, sparse: the launch is bound by DRAM
                        // traffic, where two units per thread keep more loads
                        // in flight (the subset: 0.447 -> 0.431 s); timed
                        // alone, in L2, one unit per thread looked faster
                        if (pick == LBM_LAYOUT_SPARSE && np == 0 && cn != 2) continue;
                        time_candidate(b, c, cn, 2);  // warm-up
                        const float ms = time_candidate(b, c, cn, 8);
                        if (ms < best_here) {
                            best_here = ms;
                            bn_of[cl] = cn;
                        }
                        if (!stepwise && ms < best) {
                            best = ms;
                            bl = cl;
                            bn = cn;
                        }
                    }
                    if (stepwise && o.solo != 2) {
                        float ms;
                        if (alone) {
                            time_solo(b, c, 2);  // warm-up
                            ms = time_solo(b, c, 8);
                        } else if (o.schedule == 2 && o.precision == LBM_FP32_SHIFTED) {
                            time_candidate_step(b, c, 2);
                            ms = time_candidate_step(b, c, 8);
                        } else {
                            ms = best_here;  // the persistent kernel's time
                        }
                        if (ms < best_step) {
                            best_step = ms;
                            bl = cl;
                        }
                    }
                    // Without the stepwise schedule, a lattice that fills the
                    // GPU alone may run faster without the batch (bn = 0: run
                    // it alone).  Only such lattices are candidates: timed by
                    // itself a small lattice pays every grid barrier alone,
                    // which in the batch is shared by all lattices
                    const int64_t units = cl == LBM_LAYOUT_SPARSE ? c->Nf : c->N;
                    if (np == 0 && (o.solo == 2 || (o.solo == 1 && !stepwise && units >= solo_min_units()))) {
                        time_solo(b, c, 2);  // warm-up
                        const float ms = time_solo(b, c, 8);
                        if (ms < best || o.solo == 2) {
                            best = ms;
                            bl = cl;
                            bn = 0;
                        }
                    }
                    lbm_destroy(c);
                }
                if (stepwise && o.solo != 2) bn = bn_of[bl];
                it = tuned.emplace(key, std::make_pair(bl, bn)).first;
            }
            if (lay == -1) lay = it->second.first;
            if (np == 0) np = it->second.second;
        }
        b->layout[i] = lay;
        b->npt[i] = np;
        b->solo.push_back(np == 0);
        lbm_options to = lo;
        to.layout = lay;
        lbm_ctx *c = nullptr;
        int rc = d.set >= 0 ? lbm_create(&c, d.mask, d.dims, d.set, d.tau, d.Lambda, d.force, &to)
                            : lbm_create_rates(&c, d.mask, d.dims, d.s, d.force, &to);
        if (rc != LBM_OK) return fail(rc);
        b->ctx.push_back(c);
    }
    std::vector<BatchLat> lats(n);
    int total_tiles = 0;
    size_t step_tiles = 0;
    uint32_t ngroups = 0;
    for (int i = 0; i < n; ++i) {
        lats[i] = make_lat(b->ctx[i], b->solo[i] ? 1 : b->npt[i]);
        lats[i].goff = ngroups;
        b->goff.push_back(ngroups);
        ngroups += groups_of(lats[i]);
        if (!b->solo[i]) total_tiles += ntiles_of(lats[i]);
        if (!b->solo[i] && wide_lat(lats[i])) b->wide = true;
        std::vector<Tile> ev, od;
        step_tiles_of(lats[i], i, ev, od);
        step_tiles += ev.size() + od.size();
    }
    b->max_tiles = total_tiles > 0 ? total_tiles : 1;
    b->ngroups = ngroups;
    b->max_step_tiles = (int)(step_tiles > 0 ? step_tiles : 1);
#define CKB(call)                                        \
    do {                                                 \
        cudaError_t e3 = (call);                         \
        if (e3 != cudaSuccess) return fail(launch_error(e3)); \
    } while (0)
    CKB(cudaMalloc(&b->d_lats, sizeof(BatchLat) * n));
    CKB(cudaMalloc(&b->d_tiles, sizeof(Tile) * b->max_tiles));
    CKB(cudaMalloc(&b->d_ntiles, sizeof(int)));
    CKB(cudaMalloc(&b->d_lat_tiles, sizeof(int2) * n));
    CKB(cudaMalloc(&b->d_steps, sizeof(int64_t) * n));
    CKB(cudaMalloc(&b->d_tile_part, sizeof(double) * 18 * (size_t)b->max_tiles));
    CKB(cudaMalloc(&b->d_bar, sizeof(GridBar)));
    CKB(cudaMalloc(&b->d_U, sizeof(double) * 9 * n));
    if (o.precision == LBM_FP32_SHIFTED && o.schedule == 2) {
        CKB(cudaMalloc(&b->d_step_tiles, sizeof(Tile) * (size_t)b->max_step_tiles));
        CKB(cudaMalloc(&b->d_step_part, sizeof(double) * 3 * 3 * (size_t)(ngroups > 0 ? ngroups : 1)));
        CKB(cudaMalloc(&b->d_want, (size_t)n));
    }
    CKB(cudaMallocHost(&b->h_steps, sizeof(int64_t) * n));
    CKB(cudaMallocHost(&b->h_U, sizeof(double) * 9 * n));
    CKB(cudaMallocHost(&b->h_err, sizeof(int)));
    CKB(cudaMemcpyAsync(b->d_lats, lats.data(), sizeof(BatchLat) * n, cudaMemcpyHostToDevice, b->stream));
    GridBar gb{0u, 0u, 0, o.test_skip_block};
    CKB(cudaMemcpyAsync(b->d_bar, &gb, sizeof gb, cudaMemcpyHostToDevice, b->stream));
    CKB(cudaStreamSynchronize(b->stream));
#undef CKB
    b->active.assign(n, 1);
    b->steps.assign(n, 0);
    b->status.assign(n, LBM_ENOTCONV);
    b->Ua.assign(n, NAN);
    b->Ub.assign(n, NAN);
    *out = b;
    return LBM_OK;
}

int lbm_batch_run(lbm_batch *b, double tol, int64_t *steps, int32_t *status) {
    if (!b || !(tol >= 0.0)) return LBM_EINVAL;
    if (b->failed) return LBM_ETIMEOUT;
    std::vector<BatchLat> lats(b->n);
    for (int i = 0; i < b->n; ++i) {
        lats[i] = make_lat(b->ctx[i], b->solo[i] ? 1 : b->npt[i]);
        lats[i].goff = b->goff[i];
    }
    // every lattice starts a fresh stopping-rule run; lattices that run alone
    // are not in the persistent kernel's tile table
    int nsolo = 0;
    for (int i = 0; i < b->n; ++i) {
        b->active[i] = !b->solo[i];
        nsolo += b->solo[i];
        b->status[i] = LBM_ENOTCONV;
        b->steps[i] = 0;
        b->ctx[i]->converged = b->ctx[i]->has_conv = false;
    }
    std::vector<int> drive(b->n);
    for (int i = 0; i < b->n; ++i) {
        const double *F = b->ctx[i]->F;
        int d = 0;
        for (int a = 1; a < 3; ++a)
            if (fabs(F[a]) > fabs(F[d])) d = a;
        drive[i] = d;
    }
    const int64_t K = b->opt.check_interval;
    bool dirty = true, dirty_step = true;
    int nact = b->n - nsolo;
    NvtxRange range("lbm_batch_run");
    while (nact > 0) {
        NvtxRange chunk_range("lbm batch chunk");
        cudaError_t e;
        // schedule 2: grouped multi-lattice launches per step.  Otherwise,
        // under the automatic schedule, lattices that fill the GPU alone run
        // their chunks with their own single-lattice kernels (graph-replayed)
        // and all others share one persistent launch; schedule 1 puts every
        // lattice in the persistent launch.
        const bool stepwise = b->d_step_tiles && b->opt.schedule == 2;
        std::vector<int> direct_now;
        if (!stepwise && b->opt.schedule == 0)
            for (int i = 0; i < b->n; ++i)
                if (b->active[i] && (int64_t)lats[i].units >= kDirectUnits) direct_now.push_back(i);
        if (stepwise) {
            if (dirty_step) {
                e = upload_step_tiles(b, lats);
                if (e != cudaSuccess) return launch_error(e);
                dirty_step = false;
            }
            e = enqueue_step_chunk(b);
            if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
            if (e != cudaSuccess) return launch_error(e);
            b->stepwise_chunks++;
        } else {
            if (!direct_now.empty()) {
                const int nm = b->opt.stop_rule == 1 ? 3 : 2;
                if (run_direct(b, direct_now, lats, K - nm, nm) != LBM_OK) return LBM_ECUDA;
                b->stepwise_chunks++;
            }
            if ((int)direct_now.size() < nact) {
                if (dirty) {
                    b->in_direct.assign(b->n, 0);
                    for (const int i : direct_now) b->in_direct[i] = 1;
                    e = upload_tiles(b, lats);
                    if (e != cudaSuccess) return launch_error(e);
                    dirty = false;
                }
                for (int i = 0; i < b->n; ++i) b->h_steps[i] = b->ctx[i]->steps;
                if (b->opt.use_graph && !b->gexec && !b->graph_ok) {
                    // capture the chunk once; fall back to direct launches if
                    // the cooperative launch cannot be captured
                    cudaGraph_t g = nullptr;
                    e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
                    if (e == cudaSuccess) {
                        cudaError_t ec = enqueue_chunk(b);
                        e = cudaStreamEndCapture(b->stream, &g);
                        if (ec == cudaSuccess && e == cudaSuccess &&
                            cudaGraphInstantiate(&b->gexec, g, 0) == cudaSuccess)
                            b->graph_ok = true;
                        if (g) cudaGraphDestroy(g);
                    }
                    cudaGetLastError();  // clear a failed capture
                    if (!b->graph_ok) b->opt.use_graph = 0;
                }
                if (b->graph_ok)
                    e = cudaGraphLaunch(b->gexec, b->stream);
                else
                    e = enqueue_chunk(b);
                if (e != cudaSuccess) return launch_error(e);
                b->launches += 2;
                b->persistent_chunks++;
            } else {
                *b->h_err = 0;
            }
            const int nmeas = b->opt.stop_rule == 1 ? 3 : 2;
            for (const int i : direct_now)  // their slots, after the persistent chunk's copy
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(b->h_U + 9 * (size_t)i, b->ctx[i]->d_U,
                                        sizeof(double) * 3 * nmeas, cudaMemcpyDeviceToHost,
                                        b->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
            if (e != cudaSuccess) return launch_error(e);
        }
        if (*b->h_err) {
            b->failed = true;
            return LBM_ETIMEOUT;
        }
        std::vector<char> advanced(b->n, 0);  // stepped through their own chunk graphs
        if (stepwise)
            for (const int i : b->direct) advanced[i] = 1;
        for (const int i : direct_now) advanced[i] = 1;
        for (int i = 0; i < b->n; ++i) {
            if (!b->active[i]) continue;
            lbm_ctx *c = b->ctx[i];
            if (!advanced[i]) c->steps += K;
            b->steps[i] += K;
            // slots 0, 1 (and 2 under stop rule 1) of this chunk's last steps
            const double *u = b->h_U + 9 * i;
            double m[3];
            const double *last;
            double ua, ub;
            if (b->opt.stop_rule == 1) {
                for (int a = 0; a < 3; ++a) m[a] = 0.5 * (u[3 + a] + u[6 + a]);
                ua = 0.5 * (u[drive[i]] + u[3 + drive[i]]);
                ub = m[drive[i]];
                last = u + 6;
            } else {
                for (int a = 0; a < 3; ++a) m[a] = u[3 + a];
                ua = u[drive[i]];
                ub = u[3 + drive[i]];
                last = u + 3;
            }
            b->Ua[i] = ua;
            b->Ub[i] = ub;
            c->has_conv = true;
            for (int a = 0; a < 3; ++a) c->U_conv[a] = m[a];
            int st = LBM_ENOTCONV;
            bool retire = false;
            if (!isfinite(last[0]) || !isfinite(last[1]) || !isfinite(last[2])) {
                st = LBM_EUNSTABLE;
                retire = true;
            } else if (isfinite(ua) && fabs(ub - ua) <= tol * fabs(ub)) {
                st = LBM_OK;
                retire = true;
            } else if (b->steps[i] >= b->opt.max_steps) {
                retire = true;
            }
            if (retire) {
                b->status[i] = st;
                b->active[i] = 0;
                c->converged = st == LBM_OK;
                c->has_conv = st != LBM_EUNSTABLE;
                --nact;
                dirty = dirty_step = true;
            }
        }
    }
    // lattices that run alone: the single-lattice path with the batch's rule
    for (int i = 0; i < b->n; ++i) {
        if (!b->solo[i]) continue;
        lbm_ctx *c = b->ctx[i];
        c->opt.stop_rule = b->opt.stop_rule;
        const int64_t l0 = c->launches;
        int64_t st = 0;
        const int rc = lbm_run_to_convergence(c, tol, &st);
        b->launches += c->launches - l0;
        if (rc != LBM_OK && rc != LBM_ENOTCONV && rc != LBM_EUNSTABLE) return rc;
        b->steps[i] = st;
        b->status[i] = rc;
    }
    for (int i = 0; i < b->n; ++i) {
        if (steps) steps[i] = b->steps[i];
        if (status) status[i] = b->status[i];
    }
    return LBM_OK;
}

int lbm_batch_permeability(lbm_batch *b, double *k) {
    if (!b || !k) return LBM_EINVAL;
    for (int i = 0; i < b->n; ++i) {
        int rc = b->ctx[i]->has_conv ? lbm_converged_permeability(b->ctx[i], k + 3 * i)
                                     : lbm_permeability(b->ctx[i], k + 3 * i);
        if (rc) return rc;
    }
    return LBM_OK;
}

int lbm_batch_mean_velocity(lbm_batch *b, double *U) {
    if (!b || !U) return LBM_EINVAL;
    for (int i = 0; i < b->n; ++i) {
        int rc = lbm_mean_velocity(b->ctx[i], U + 3 * i);
        if (rc) return rc;
    }
    return LBM_OK;
}

int lbm_batch_config(lbm_batch *b, int32_t *layout, int32_t *npt) {
    if (!b) return LBM_EINVAL;
    const bool own = b->opt.schedule == 0 || (b->opt.schedule == 2 && b->d_step_tiles);
    for (int i = 0; i < b->n; ++i) {
        if (layout) layout[i] = b->layout[i];
        if (npt) {
            // a lattice that runs its chunks on its own kernels is in no tile
            const lbm_ctx *c = b->ctx[i];
            const int64_t units = b->layout[i] == LBM_LAYOUT_SPARSE ? c->Nf : c->N;
            npt[i] = own && units >= kDirectUnits ? 0 : b->npt[i];
        }
    }
    return LBM_OK;
}

lbm_ctx *lbm_batch_lattice(lbm_batch *b, int32_t i) {
    if (!b || i < 0 || i >= b->n) return nullptr;
    return b->ctx[i];
}

int64_t lbm_batch_kernel_launches(const lbm_batch *b) { return b ? b->launches : -1; }

int lbm_batch_schedule_counts(const lbm_batch *b, int64_t *stepwise, int64_t *persistent) {
    if (!b) return LBM_EINVAL;
    if (stepwise) *stepwise = b->stepwise_chunks;
    if (persistent) *persistent = b->persistent_chunks;
    return LBM_OK;
}

}  // extern "C"
