// Stream-collide kernels of the D3Q19-MRT solver and the kernels that read
// or write its state.
//
// One thread updates one fluid node per launch: it gathers the 19 streamed
// populations (pull scheme, eq. LBE; halfway bounceback where the upstream
// voxel is solid), runs the MRT collision with Guo forcing in registers
// (lbm_collide.cuh), stores the 19 post-collision populations, and, on
// launches that measure, adds its shifted velocity to a per-block FP64
// partial sum.  Populations are structure-of-arrays, slot i of node n at
// i*N + n (N = nodes, or fluid nodes for the sparse layout), so each warp's
// access to a slot is one contiguous run.
//
// Layouts
//  AB      pull from array `src` into array `dst` (two arrays).
//  AA      one array.  An even step reads a node's own slots and writes the
//          post-collision value of direction opp(j) back into slot j; an odd
//          step reads slot opp(j) of the upstream neighbour x - c_j (slot j of
//          the node itself if that neighbour is solid) and writes the
//          post-collision value of direction opp(j) back to the same place.
//          Each thread therefore reads and writes exactly the same 19
//          locations, so no two threads touch one location within a step.
//  SPARSE  the AA pattern over the fluid list, neighbours from a table.
#include <math.h>
#include <string.h>

#include "lbm_step.cuh"

namespace lbm {

// ---------------------------------------------------------------- helpers

// Per-block partial sums of the momenta into red.partials[3 * blockIdx.x ..].
template <typename C>
__device__ __forceinline__ void block_reduce_velocity(C jx, C jy, C jz, bool fluid,
                                                      const Reduce &red) {
    block_momentum_sum<C>(jx, jy, jz, fluid, red.partials + 3 * (size_t)blockIdx.x, red.flag);
}

// ---------------------------------------------------------------- AB pull

template <typename S, int K>
__global__ void __launch_bounds__(256) k_ab(const S *__restrict__ src, S *__restrict__ dst,
                                            const uint32_t *__restrict__ lw, Dims d,
                                            Collide<typename Store<S>::C> p, float ld_scale,
                                            float st_scale, Reduce red) {
    using C = typename Store<S>::C;
    const uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t w = n < d.N ? lw[n] : SOLID_BIT;
    const bool fluid = !(w & NOT_FLUID);
    C jx = C(0), jy = C(0), jz = C(0);
    if (fluid || (w & BBNODE_BIT)) {
        DenseNode nd;
        nd.init(n, d);
        const uint64_t lim = (uint64_t)Q * d.N;
        C g[Q];
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            const size_t at = j == 0 ? (size_t)n
                              : (w & (1u << j)) ? (size_t)opp(j) * d.N + n
                                                : (size_t)j * d.N + nd.up(j);
            g[j] = in_range(at, lim, red.flag) ? Store<S>::ld(src + at, ld_scale) : C(0);
        }
        if (fluid) {
            collide_as<K, C>(g, p, jx, jy, jz);
#pragma unroll
            for (int i = 0; i < Q; ++i) Store<S>::st(dst + (size_t)i * d.N + n, g[i], st_scale);
        } else {
            // full-way bounceback voxel: each population streamed in leaves
            // along the opposite link in the next step
#pragma unroll
            for (int i = 0; i < Q; ++i) Store<S>::st(dst + (size_t)i * d.N + n, g[opp(i)], st_scale);
        }
    }
    if (red.partials) block_reduce_velocity<C>(jx, jy, jz, fluid, red);
}

// ------------------------------------------------------ AA, dense and sparse

template <typename S, bool ODD, int K>
__global__ void __launch_bounds__(256) k_aa(S *A, const uint32_t *__restrict__ lw, Dims d,
                                            Collide<typename Store<S>::C> p, float ld_scale,
                                            float st_scale, Reduce red) {
    using C = typename Store<S>::C;
    const uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t w = n < d.N ? lw[n] : SOLID_BIT;
    C jx = C(0), jy = C(0), jz = C(0);
    const bool fluid = aa_dense_update<S, ODD, Store<S>, K>(A, n, w, d, p, ld_scale, st_scale, jx,
                                                            jy, jz, red.flag);
    if (red.partials) block_reduce_velocity<C>(jx, jy, jz, fluid, red);
}

// Minimum resident blocks per SM for the sparse stream-collide (caps the
// registers per thread; more resident warps hide the odd step's dependent
// index loads).
#ifndef LBM_SPARSE_MIN_BLOCKS
#define LBM_SPARSE_MIN_BLOCKS 3
#endif
#ifndef LBM_SPARSE_MIN_BLOCKS_EVEN
#define LBM_SPARSE_MIN_BLOCKS_EVEN 3
#endif

// One node per thread: the even steps of FP64 storage (the FP32 and FP16
// steps use the tiled kernels below).  Idx: type of the flat population
// offsets; uint32_t whenever 19 * Nf < 2^32.
template <typename S, bool ODD, typename Idx, int K>
__global__ void __launch_bounds__(256, sizeof(S) == 8 ? 2
                                       : (ODD ? LBM_SPARSE_MIN_BLOCKS : LBM_SPARSE_MIN_BLOCKS_EVEN))
    k_sparse(S *A, SparseMap m, uint32_t Nf, Collide<typename Store<S>::C> p, float ld_scale,
             float st_scale, Reduce red) {
    using C = typename Store<S>::C;
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    const bool fluid = k < Nf;
    C jx = C(0), jy = C(0), jz = C(0);
    if (fluid) {
        const uint2 nb = ODD ? __ldg(m.nb + k) : make_uint2(0u, 0u);
        aa_sparse_update<S, ODD, Idx, Store<S>, K>(A, m, Nf, k, nb, p, ld_scale, st_scale, jx, jy, jz);
    }
    if (red.partials) block_reduce_velocity<C>(jx, jy, jz, fluid, red);
}

// Odd steps: NPT nodes per thread.  A block takes a tile of 256 * NPT
// consecutive fluid nodes and thread t the nodes first + t, first + t + 256,
// ...; each node's {node index, bounceback bits} record is loaded one node
// ahead, so that dependent fetch overlaps the previous node's gathers and
// collision.  (A persistent grid-stride version of the same loop hides the
// index chain as well but streams about a fifth slower; four nodes per
// thread measured best.)
#ifndef LBM_SPARSE_ODD_NPT
#define LBM_SPARSE_ODD_NPT 4
#endif

// RED: also the per-256-node partial momentum sums of a measuring step
// (partial g covers fluid nodes 256 g .. 256 g + 255, as in k_sparse).
template <typename S, typename Idx, int NPT, int K, bool RED>
__global__ void __launch_bounds__(256, sizeof(S) == 8 ? 2 : LBM_SPARSE_MIN_BLOCKS)
    k_sparse_odd_t(S *A, SparseMap m, uint32_t Nf, Collide<typename Store<S>::C> p,
                   float ld_scale, float st_scale, Reduce red) {
    using C = typename Store<S>::C;
    __shared__ double wsum[RED ? NPT : 1][8][3];  // RED: warp sums of each group
    uint32_t k = blockIdx.x * (256u * NPT) + threadIdx.x;
    uint2 nxt = k < Nf ? __ldg(m.nb + k) : make_uint2(0u, 0u);
    int groups = 0;
#pragma unroll 1
    for (int r = 0; r < NPT; ++r, k += 256u) {
        const uint32_t group = blockIdx.x * (uint32_t)NPT + (uint32_t)r;
        if (RED ? group * 256u >= Nf : k >= Nf) break;  // block-uniform when RED
        const bool valid = k < Nf;
        const uint2 cur = nxt;
        if (r + 1 < NPT && k + 256u < Nf) nxt = __ldg(m.nb + k + 256u);
        C jx = C(0), jy = C(0), jz = C(0);
        if (valid)
            aa_sparse_update<S, true, Idx, Store<S>, K>(A, m, Nf, k, cur, p, ld_scale, st_scale,
                                                        jx, jy, jz);
        if (RED) warp_momentum_store<C>(jx, jy, jz, valid, wsum[RED ? r : 0], red.flag);
        ++groups;
    }
    if (RED) {  // one synchronisation for all of the tile's groups
        __syncthreads();
        if ((int)threadIdx.x < 3 * groups) {
            const int r = threadIdx.x / 3, a = threadIdx.x % 3;
            red.partials[3 * (size_t)(blockIdx.x * (uint32_t)NPT + (uint32_t)r) + a] =
                group_momentum_total(wsum[r], a);
        }
    }
}

// Odd steps, FP32 or FP16 storage, 32-bit offsets, Lx < 2^13: the tiling of
// k_sparse_odd_t (four nodes per thread, the next node's record loaded
// ahead) with the index arithmetic of odd_lean_locations (no division, no
// wrap test, slot offsets from the parameter bank).  Bitwise the results of
// k_sparse_odd_t; at 512^3 1% faster with FP32 storage and 6% with FP16.
#ifndef LBM_ODD_LEAN
#define LBM_ODD_LEAN 1  // 0: FP32/FP16 odd steps through k_sparse_odd_t as well
#endif
template <typename S, int NPT, int K, bool RED>
__global__ void __launch_bounds__(256, LBM_SPARSE_MIN_BLOCKS)
    k_sparse_odd_l(S *A, OddMap o, uint32_t Nf, Collide<typename Store<S>::C> p, float ld_scale,
                   float st_scale, Reduce red) {
    using C = typename Store<S>::C;
    // FP16 storage: p is scaled_collide's and the halves are collided as
    // stored; ld_scale (2^-S) only unscales the measured momentum
    constexpr bool kRaw = sizeof(S) == 2;
    __shared__ double wsum[RED ? NPT : 1][8][3];  // RED: warp sums of each group
    uint32_t k = blockIdx.x * (256u * NPT) + threadIdx.x;
    uint2 nxt = k < Nf ? __ldg(o.rec + k) : make_uint2(0u, 0u);
    const uint64_t lim = (uint64_t)Q * Nf;
    int groups = 0;
#pragma unroll 1
    for (int r = 0; r < NPT; ++r, k += 256u) {
        const uint32_t group = blockIdx.x * (uint32_t)NPT + (uint32_t)r;
        if (RED ? group * 256u >= Nf : k >= Nf) break;  // block-uniform when RED
        const bool valid = k < Nf;
        const uint2 cur = nxt;
        if (r + 1 < NPT && k + 256u < Nf) nxt = __ldg(o.rec + k + 256u);
        C jx = C(0), jy = C(0), jz = C(0);
        if (valid) {
            uint32_t loc[Q];
            odd_lean_locations(o, k, cur, loc);
            C g[Q];
#pragma unroll
            for (int j = 0; j < Q; ++j) {
                if (!in_range(loc[j], lim, o.flag))
                    g[j] = C(0);
                else if constexpr (kRaw)
                    g[j] = __half2float(A[loc[j]]);
                else
                    g[j] = Store<S>::ld(A + loc[j], ld_scale);
            }
            collide_as<K, C>(g, p, jx, jy, jz);
#pragma unroll
            for (int j = 0; j < Q; ++j) {
                if (!in_range(loc[j], lim, o.flag)) continue;
                if constexpr (kRaw)
                    A[loc[j]] = __float2half_rn(g[opp(j)]);
                else
                    Store<S>::st(A + loc[j], g[opp(j)], st_scale);
            }
            if (kRaw) {  // the measured momentum in unscaled units
                jx = __fmul_rn(jx, ld_scale);
                jy = __fmul_rn(jy, ld_scale);
                jz = __fmul_rn(jz, ld_scale);
            }
        }
        if (RED) warp_momentum_store<C>(jx, jy, jz, valid, wsum[RED ? r : 0], red.flag);
        ++groups;
    }
    if (RED) {  // one synchronisation for all of the tile's groups
        __syncthreads();
        if ((int)threadIdx.x < 3 * groups) {
            const int r = threadIdx.x / 3, a = threadIdx.x % 3;
            red.partials[3 * (size_t)(blockIdx.x * (uint32_t)NPT + (uint32_t)r) + a] =
                group_momentum_total(wsum[r], a);
        }
    }
}

// Even steps, FP32 or FP16 storage: two nodes per thread, 256 apart, with
// the loads of both issued before either collision.
// At two blocks per SM this keeps about a third more bytes in flight than one
// node per thread at three blocks per SM (1.31 -> 1.25 ms at 512^3).
template <typename S, int K, bool RED>
__global__ void __launch_bounds__(256, 2)
    k_sparse_even_x2(S *A, uint32_t Nf, Collide<typename Store<S>::C> p, float ld_scale,
                     float st_scale, Reduce red) {
    using C = typename Store<S>::C;
    const uint32_t k0 = blockIdx.x * 512u + threadIdx.x, k1 = k0 + 256u;
    const bool v0 = k0 < Nf, v1 = k1 < Nf;
    C g0[Q], g1[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) g0[j] = v0 ? Store<S>::ld(A + (uint32_t)j * Nf + k0, ld_scale) : C(0);
#pragma unroll
    for (int j = 0; j < Q; ++j) g1[j] = v1 ? Store<S>::ld(A + (uint32_t)j * Nf + k1, ld_scale) : C(0);
    C jx0 = C(0), jy0 = C(0), jz0 = C(0), jx1 = C(0), jy1 = C(0), jz1 = C(0);
    if (v0) {
        collide_as<K, C>(g0, p, jx0, jy0, jz0);
#pragma unroll
        for (int j = 0; j < Q; ++j) Store<S>::st(A + (uint32_t)j * Nf + k0, g0[opp(j)], st_scale);
    }
    if (v1) {
        collide_as<K, C>(g1, p, jx1, jy1, jz1);
#pragma unroll
        for (int j = 0; j < Q; ++j) Store<S>::st(A + (uint32_t)j * Nf + k1, g1[opp(j)], st_scale);
    }
    if (RED) {  // partials 2b and 2b + 1 (nodes 256 g .. 256 g + 255, as in k_sparse)
        __shared__ double wsum[2][8][3];
        warp_momentum_store<C>(jx0, jy0, jz0, v0, wsum[0], red.flag);
        warp_momentum_store<C>(jx1, jy1, jz1, v1, wsum[1], red.flag);
        __syncthreads();
        const int ng = (2 * blockIdx.x + 1) * 256u < Nf ? 2 : 1;
        if ((int)threadIdx.x < 3 * ng) {
            const int r = threadIdx.x / 3, a = threadIdx.x % 3;
            red.partials[3 * (size_t)(2 * blockIdx.x + r) + a] = group_momentum_total(wsum[r], a);
        }
    }
}

// Even steps, FP16 storage: four nodes per thread, 256 apart, all 76 loads
// issued before the first collision.  The stored halves of two nodes are
// packed into one 32-bit register (half2), so the four nodes' loads fit the
// registers the two-node FP32 kernel uses, and a warp keeps as many bytes
// in flight as that kernel does (two-byte values need twice the loads).
// p is scaled_collide's: the halves are collided as stored, and inv (2^-S)
// only brings the measured momentum back to unscaled units.
#ifndef LBM_EVEN_H4
#define LBM_EVEN_H4 1  // 0: FP16 even steps through k_sparse_even_x2 as well
#endif
#ifndef LBM_EVEN_P2
#define LBM_EVEN_P2 1  // 0: FP16 plain even steps through k_sparse_even_h4 also for even N_f
#endif
template <int K, bool RED>
__global__ void __launch_bounds__(256, 2)
    k_sparse_even_h4(__half *A, uint32_t Nf, Collide<float> p, float inv, Reduce red) {
    const uint32_t k0 = blockIdx.x * 1024u + threadIdx.x;
    __half2 h01[Q], h23[Q];  // (node 0, node 1) and (node 2, node 3) of this thread
    const __half z = __float2half_rn(0.f);
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        const __half *a = A + (uint32_t)j * Nf;
        h01[j] = __halves2half2(k0 < Nf ? a[k0] : z, k0 + 256u < Nf ? a[k0 + 256u] : z);
        h23[j] = __halves2half2(k0 + 512u < Nf ? a[k0 + 512u] : z,
                                k0 + 768u < Nf ? a[k0 + 768u] : z);
    }
    __shared__ double wsum[RED ? 4 : 1][8][3];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const uint32_t k = k0 + 256u * r;
        const bool v = k < Nf;
        float g[Q];
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            const __half2 h = r < 2 ? h01[j] : h23[j];
            g[j] = __half2float((r & 1) ? __high2half(h) : __low2half(h));
        }
        float jx = 0.f, jy = 0.f, jz = 0.f;
        if (v) {
            collide_as<K, float>(g, p, jx, jy, jz);
#pragma unroll
            for (int j = 0; j < Q; ++j) A[(uint32_t)j * Nf + k] = __float2half_rn(g[opp(j)]);
        }
        if (RED)
            warp_momentum_store<float>(__fmul_rn(jx, inv), __fmul_rn(jy, inv), __fmul_rn(jz, inv), v,
                                       wsum[RED ? r : 0], red.flag);
    }
    if (RED) {  // partials 4b .. 4b + 3 (nodes 256 g .. 256 g + 255, as in k_sparse)
        __syncthreads();
        const uint32_t g0 = 4u * blockIdx.x;
        int ng = 0;
        while (ng < 4 && (g0 + (uint32_t)ng) * 256u < Nf) ++ng;
        if ((int)threadIdx.x < 3 * ng) {
            const int r = threadIdx.x / 3, a = threadIdx.x % 3;
            red.partials[3 * (size_t)(g0 + (uint32_t)r) + a] = group_momentum_total(wsum[r], a);
        }
    }
}

// Even steps, FP16 storage, N_f even (so every slot starts on a 4-byte
// boundary), plain steps: the adjacent nodes 2m and 2m + 1 share one 32-bit
// word per slot.  A thread loads and stores such a pair with one access per
// slot and packs the pair's two results with one conversion, which takes
// two of the six instructions per stored value of k_sparse_even_h4 away.
// Two pairs per thread, 256 pairs apart (1024 nodes per block).  Measuring
// steps keep k_sparse_even_h4, whose warps sum the nodes in the order of
// every other kernel.  p is scaled_collide's (halves collided as stored).
template <int K>
__global__ void __launch_bounds__(256, 2)
    k_sparse_even_p2(__half2 *A, uint32_t Nf, Collide<float> p) {
    const uint32_t np = Nf / 2u;  // node pairs per slot
    const uint32_t q0 = blockIdx.x * 512u + threadIdx.x, q1 = q0 + 256u;
    const bool v0 = q0 < np, v1 = q1 < np;
    const __half2 z = __float2half2_rn(0.f);
    __half2 w0[Q], w1[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        w0[j] = v0 ? A[(uint32_t)j * np + q0] : z;
        w1[j] = v1 ? A[(uint32_t)j * np + q1] : z;
    }
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        if (!(t ? v1 : v0)) continue;
        const uint32_t q = t ? q1 : q0;
        float ga[Q], gb[Q], jx, jy, jz;
#pragma unroll
        for (int j = 0; j < Q; ++j) ga[j] = __low2float(t ? w1[j] : w0[j]);
        collide_as<K, float>(ga, p, jx, jy, jz);
#pragma unroll
        for (int j = 0; j < Q; ++j) gb[j] = __high2float(t ? w1[j] : w0[j]);
        collide_as<K, float>(gb, p, jx, jy, jz);
#pragma unroll
        for (int j = 0; j < Q; ++j) A[(uint32_t)j * np + q] = __floats2half2_rn(ga[opp(j)], gb[opp(j)]);
    }
}

// ------------------------------------------------------- reduction finalise

// Fixed-order sum of the per-block partials: thread t adds blocks t, t+T, ...
// in order, then a fixed shared-memory tree.  out[a] = sum / N_total.
__global__ void __launch_bounds__(1024) k_finalize(const double *__restrict__ partials, int nblk,
                                                   double inv_total, double *out) {
    __shared__ double sm[3][1024];
    double acc[3] = {0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblk; b += blockDim.x)
#pragma unroll
        for (int a = 0; a < 3; ++a) acc[a] += partials[3 * (size_t)b + a];
#pragma unroll
    for (int a = 0; a < 3; ++a) sm[a][threadIdx.x] = acc[a];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
#pragma unroll
            for (int a = 0; a < 3; ++a) sm[a][threadIdx.x] += sm[a][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < 3) out[threadIdx.x] = sm[threadIdx.x][0] * inv_total;
}

// ------------------------------------------------ state readers and writers

// Where the current state keeps, for unit u (node or fluid index), the
// streamed population of direction j (kind 0) or the post-collision
// population of direction opp(j) (kind 1).
struct StateView {
    int layout;      // LBM_LAYOUT_*
    int parity;      // steps % 2 (AA, SPARSE)
    uint32_t units;  // N (dense) or Nf (sparse)
    const uint32_t *lw;
    SparseMap sm;
    Dims d;
    // bounds-check build: a location outside the 19 * units slots
    __device__ __forceinline__ bool ok(size_t at) const { return in_range(at, (uint64_t)Q * units, sm.flag); }
};

struct UnitNode {
    DenseNode d;
    SparseNode s;
};

// Returns the flat offset for unit u, direction j.  For AB, kind 0 reads the
// pull location in the current array and kind 1 the node's own slot
// (holding f*_opp(j) for slot opp(j)).
__device__ __forceinline__ size_t state_loc(const StateView &v, uint32_t u, int j, int kind,
                                            uint32_t w, const UnitNode &un) {
    const DenseNode &nd = un.d;
    if (v.layout == LBM_LAYOUT_AB) {
        if (kind == 1) return (size_t)opp(j) * v.units + u;  // f*_opp(j) lives in slot opp(j)
        if (j == 0) return u;
        if (w & (1u << j)) return (size_t)opp(j) * v.units + u;
        return (size_t)j * v.units + nd.up(j);
    }
    // AA / SPARSE: streamed state sits at the parity's pattern, the
    // post-collision state (direction opp(j) at location j) at the other one.
    const bool odd = (kind == 0) ? (v.parity == 1) : (v.parity == 0);
    if (!odd || j == 0 || (w & (1u << j))) return (size_t)j * v.units + u;
    if (v.layout == LBM_LAYOUT_AA) return (size_t)opp(j) * v.units + nd.up(j);
    return (size_t)opp(j) * v.units + un.s.up(j, v.sm);
}

__device__ __forceinline__ bool state_unit(const StateView &v, uint32_t u, uint32_t &node,
                                           uint32_t &w, UnitNode &un) {
    node = u;
    if (v.layout == LBM_LAYOUT_SPARSE) {
        un.s.init(u, v.sm);
        w = un.s.bits;
        return true;
    }
    w = v.lw[u];
    if (w & NOT_FLUID) return false;
    un.d.init(u, v.d);
    return true;
}

// Streamed-state velocity u = sum c f + F/2 per unit; writes the field
// (dense node order, indexed through fidx for the sparse layout) and/or
// block partials for the mean.
template <typename S>
__global__ void __launch_bounds__(256) k_velocity(const S *A, StateView v,
                                                  const int32_t *__restrict__ fidx, double Fx,
                                                  double Fy, double Fz, float ld_scale,
                                                  double *u_out, Reduce red) {
    using C = typename Store<S>::C;
    const uint32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    bool fluid = false;
    double jx = 0.0, jy = 0.0, jz = 0.0;
    if (u < v.units) {
        uint32_t node, w;
        UnitNode nd;
        fluid = state_unit(v, u, node, w, nd);
        if (fluid) {
#pragma unroll
            for (int j = 1; j < Q; ++j) {
                const size_t at = state_loc(v, u, j, 0, w, nd);
                double gj = v.ok(at) ? (double)Store<S>::ld(A + at, ld_scale) : 0.0;
                jx += cx(j) * gj;
                jy += cy(j) * gj;
                jz += cz(j) * gj;
            }
            jx += 0.5 * Fx;
            jy += 0.5 * Fy;
            jz += 0.5 * Fz;
        }
        if (u_out) {
            size_t N = v.d.N;
            size_t out = v.layout == LBM_LAYOUT_SPARSE ? (size_t)fidx[u] : (size_t)u;
            u_out[out] = jx;
            u_out[N + out] = jy;
            u_out[2 * N + out] = jz;
        }
    }
    if (red.partials) block_reduce_velocity<double>(jx, jy, jz, fluid, red);
}

// Mean-velocity partials alone (no field export), FP32 or FP16 storage: the
// per-node momentum in float, summed per block as in the stepping kernels.
// SP: sparse layout, with its streamed values read as the odd step forms
// them (even parity: the node's own slots; odd parity: the interior
// upstream formulas, clamped, with the x faces redone).  FP64 arithmetic is
// scarce on this GPU; the FP64 k_velocity took 9.3 ms at 512^3.
template <typename S, bool SP>
__global__ void __launch_bounds__(256) k_velocity_sum(const S *A, StateView v, float Fx, float Fy,
                                                      float Fz, float ld_scale, Reduce red) {
    using C = typename Store<S>::C;
    const uint32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    bool fluid = false;
    C jx = C(0), jy = C(0), jz = C(0);
    if (u < v.units) {
        C g[Q];
        if (SP) {
            fluid = true;
            if (v.parity == 0) {
#pragma unroll
                for (int j = 1; j < Q; ++j) g[j] = Store<S>::ld(A + (size_t)j * v.units + u, ld_scale);
            } else {
                SparseNode sn;
                sn.init(u, v.sm);
#pragma unroll
                for (int j = 1; j < Q; ++j) {
                    uint32_t up = sn.up_interior(j);
                    if (cx(j) != 0) up = min(up, v.units - 1u);  // in bounds; x faces redone below
                    const size_t at = (sn.bits & (1u << j)) ? (size_t)j * v.units + u
                                                            : (size_t)opp(j) * v.units + up;
                    g[j] = v.ok(at) ? Store<S>::ld(A + at, ld_scale) : C(0);
                }
                if (sn.xlo || sn.xhi) {
#pragma unroll
                    for (int j = 1; j < Q; ++j)
                        if (cx(j) != 0 && !(sn.bits & (1u << j))) {
                            const size_t at = (size_t)opp(j) * v.units + sn.up(j, v.sm);
                            g[j] = v.ok(at) ? Store<S>::ld(A + at, ld_scale) : C(0);
                        }
                }
            }
        } else {
            uint32_t node, w;
            UnitNode nd;
            fluid = state_unit(v, u, node, w, nd);
            if (fluid) {
#pragma unroll
                for (int j = 1; j < Q; ++j) {
                    const size_t at = state_loc(v, u, j, 0, w, nd);
                    g[j] = v.ok(at) ? Store<S>::ld(A + at, ld_scale) : C(0);
                }
            }
        }
        if (fluid) {
#pragma unroll
            for (int j = 1; j < Q; ++j) {
                jx += C(cx(j)) * g[j];
                jy += C(cy(j)) * g[j];
                jz += C(cz(j)) * g[j];
            }
            jx += C(0.5) * Fx;
            jy += C(0.5) * Fy;
            jz += C(0.5) * Fz;
        }
    }
    block_momentum_sum<C>(jx, jy, jz, fluid, red.partials + 3 * (size_t)blockIdx.x, red.flag);
}

// Export of the post-collision state as unshifted FP64 f[19][N] (dense node
// order).  Solid nodes are left to the caller (who fills w_i).
template <typename S>
__global__ void __launch_bounds__(256) k_export(const S *A, StateView v,
                                                const int32_t *__restrict__ fidx, float ld_scale,
                                                double *f) {
    const uint32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= v.units) return;
    uint32_t node, w;
    UnitNode nd;
    if (!state_unit(v, u, node, w, nd)) return;
    const size_t out = v.layout == LBM_LAYOUT_SPARSE ? (size_t)fidx[u] : (size_t)u;
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        const size_t at = state_loc(v, u, j, 1, w, nd);
        double gv = v.ok(at) ? (double)Store<S>::ld(A + at, ld_scale) : 0.0;
        f[(size_t)opp(j) * v.d.N + out] = gv + weight(opp(j));
    }
}

template <typename S>
__global__ void __launch_bounds__(256) k_import(S *A, StateView v, const int32_t *__restrict__ fidx,
                                                float st_scale, const double *f) {
    const uint32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= v.units) return;
    uint32_t node, w;
    UnitNode nd;
    if (!state_unit(v, u, node, w, nd)) return;
    const size_t in = v.layout == LBM_LAYOUT_SPARSE ? (size_t)fidx[u] : (size_t)u;
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        double fv = f[(size_t)opp(j) * v.d.N + in] - weight(opp(j));
        const size_t at = state_loc(v, u, j, 1, w, nd);
        if (v.ok(at)) Store<S>::st(A + at, (typename Store<S>::C)fv, st_scale);
    }
}

// Post-collision populations at listed node indices, f[k][19] unshifted.
// Sparse layouts find the fluid index by binary search in the sorted list.
template <typename S>
__global__ void __launch_bounds__(256) k_export_at(const S *A, StateView v,
                                                   const int32_t *__restrict__ fidx,
                                                   const int64_t *__restrict__ nodes, int count,
                                                   float ld_scale, double *f) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    const uint32_t node = (uint32_t)nodes[k];
    uint32_t unit = node;
    bool fluid;
    uint32_t w = 0;
    UnitNode nd;
    if (v.layout == LBM_LAYOUT_SPARSE) {
        int lo = 0, hi = (int)v.units - 1;
        fluid = false;
        while (lo <= hi) {
            const int mid = (lo + hi) >> 1;
            const uint32_t mv = (uint32_t)fidx[mid];
            if (mv == node) {
                fluid = true;
                unit = (uint32_t)mid;
                break;
            }
            if (mv < node) lo = mid + 1;
            else hi = mid - 1;
        }
        if (fluid) {
            nd.s.init(unit, v.sm);
            w = nd.s.bits;
        }
    } else {
        w = v.lw[node];
        fluid = !(w & NOT_FLUID);
        if (fluid) nd.d.init(node, v.d);
    }
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        double val = weight(opp(j));
        if (fluid) {
            const size_t at = state_loc(v, unit, j, 1, w, nd);
            if (v.ok(at)) val += (double)Store<S>::ld(A + at, ld_scale);
        }
        f[(size_t)k * Q + opp(j)] = val;
    }
}

// ---------------------------------------------------------------- launchers

static inline unsigned nblocks(uint64_t units, int bs) { return (unsigned)((units + bs - 1) / bs); }

// 32-bit population offsets: whenever 19 * Nf < 2^32, unless the context
// asked for 64-bit offsets (lbm_options.index_width = 64).
static inline bool narrow_index(const lbm_ctx *c) {
    return c->opt.index_width != 64 && 19 * (uint64_t)c->Nf < (uint64_t(1) << 32);
}

// The kernel parameters of k_sparse_odd_l (see OddMap).
OddMap odd_map(const lbm_ctx *c) {
    OddMap o;
    memset(&o, 0, sizeof o);
    o.rec = c->d_orec;
    o.Wr = (uint32_t)c->Wr;
    o.Lx = (uint32_t)c->Lx;
    o.rwp = c->d_rwp;
    o.rse0 = c->d_rse;
    o.nprows = (uint32_t)(c->Ly + 2) * (uint32_t)(c->Lz + 2);
    o.flag = c->d_flag;
    for (int s = 0; s < 9; ++s) {
        // neighbour row slot s of padded row p is p + dy + (Ly + 2) dz
        const int dy = s < 8 ? slot_dy(s) : 0, dz = s < 8 ? slot_dz(s) : 0;
        o.roff[s] = dy + (c->Ly + 2) * dz;
        o.rse[s] = (const int2 *)((uintptr_t)c->d_rse + (intptr_t)o.roff[s] * (intptr_t)sizeof(int2));
        if (s < 8)
            o.rws[s] = (const RowWord *)((uintptr_t)c->d_rwp +
                                         (intptr_t)o.roff[s] * c->Wr * (intptr_t)sizeof(RowWord));
    }
    for (int j = 0; j < Q; ++j) o.slot[j] = (uint32_t)j * (uint32_t)c->Nf;
    return o;
}

SparseMap sparse_map(const lbm_ctx *c) {
    SparseMap m;
    m.fidx = c->d_fidx;
    m.bb = c->d_bb;
    m.nb = c->d_nb;
    m.rw = c->d_rw;
    m.rstart = c->d_rstart;
    m.Lx = c->Lx;
    m.Ly = c->Ly;
    m.Lz = c->Lz;
    m.Wr = c->Wr;
    m.mLx = div_magic((uint32_t)c->Lx);
    m.mLy = div_magic((uint32_t)c->Ly);
    m.flag = c->d_flag;
    return m;
}

// Fluid nodes per thread of the odd step's lean kernel for this lattice:
// four (the next record loaded ahead, fewest blocks) while the grid still
// gives every SM its resident blocks, else two, else one, so that a small
// lattice keeps all SMs busy.  FP32 per launch: 64^3 Boolean (104k fluid
// nodes) 12.3 us with four per thread, 9.3 us with one; from 128^3 up four
// are best (256^3: 223, 228 and 241 us with four, two and one).
template <typename S, int K>
static int odd_nodes_per_thread(lbm_ctx *c) {
    if (c->odd_npt) return c->odd_npt;
    int sms = 0, per = 0;
    // a failed query falls back to defaults; its error is cleared, and only
    // then, so that an earlier launch's error stays visible to the caller
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
        sms = 0;
        cudaGetLastError();
    }
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sparse_odd_l<S, 4, K, false>, 256,
                                                      0) != cudaSuccess) {
        per = 0;
        cudaGetLastError();
    }
    const int64_t slots = (int64_t)(sms > 0 ? sms : 1) * (per > 0 ? per : LBM_SPARSE_MIN_BLOCKS);
    int best = 1;
    for (const int n : {4, 2}) {
        if ((c->Nf + 256 * n - 1) / (256 * n) >= slots) {
            best = n;
            break;
        }
    }
    c->odd_npt = best;
    return best;
}

template <typename S, int NPT, int K>
static void launch_odd_lean(lbm_ctx *c, bool reduce, const OddMap &o, S *A, uint32_t Nf,
                            const Collide<typename Store<S>::C> &p, float lds, float sts,
                            const Reduce &red) {
    const unsigned tg = (unsigned)((Nf + 256u * NPT - 1) / (256u * NPT));
    Collide<typename Store<S>::C> pk = p;
    if constexpr (sizeof(S) == 2) pk = scaled_collide(p, sts);
    if (reduce)
        k_sparse_odd_l<S, NPT, K, true><<<tg, 256, 0, c->stream>>>(A, o, Nf, pk, lds, sts, red);
    else
        k_sparse_odd_l<S, NPT, K, false><<<tg, 256, 0, c->stream>>>(A, o, Nf, pk, lds, sts, red);
}

template <typename S, int K>
int launch_step_k(lbm_ctx *c, bool reduce, const Collide<typename Store<S>::C> &p) {
    const int bs = c->opt.block_size;
    const float lds = c->fp16_scale > 0.f ? 1.0f / c->fp16_scale : 1.0f;
    const float sts = c->fp16_scale > 0.f ? c->fp16_scale : 1.0f;
    Dims d{c->Lx, c->Ly, c->Lz, (uint32_t)c->N};
    Reduce red{reduce ? c->d_partials : nullptr, c->d_flag};
    const bool odd = (c->steps & 1) != 0;
    unsigned grid;
    switch (c->opt.layout) {
    case LBM_LAYOUT_AB:
        grid = nblocks(c->N, bs);
        k_ab<S, K><<<grid, bs, 0, c->stream>>>((const S *)c->d_pop[c->cur], (S *)c->d_pop[1 - c->cur],
                                            c->d_lw, d, p, lds, sts, red);
        c->cur = 1 - c->cur;
        break;
    case LBM_LAYOUT_AA:
        grid = nblocks(c->N, bs);
        if (odd)
            k_aa<S, true, K><<<grid, bs, 0, c->stream>>>((S *)c->d_pop[0], c->d_lw, d, p, lds, sts, red);
        else
            k_aa<S, false, K><<<grid, bs, 0, c->stream>>>((S *)c->d_pop[0], c->d_lw, d, p, lds, sts, red);
        break;
    default:
        grid = nblocks(c->Nf, bs);
        if (grid == 0) break;
        // measuring steps write one partial per 256 fluid nodes
        const unsigned groups = (unsigned)((c->Nf + 255) / 256);
        if constexpr (sizeof(S) == 2 && LBM_EVEN_H4) {
            if (!odd && narrow_index(c)) {
                const unsigned g4 = (unsigned)((c->Nf + 1023) / 1024);
                const Collide<float> ps = scaled_collide(p, sts);
                if (!reduce && LBM_EVEN_P2 && c->Nf % 2 == 0) {
                    const unsigned gp = (unsigned)((c->Nf / 2 + 511) / 512);
                    k_sparse_even_p2<K><<<gp, 256, 0, c->stream>>>((__half2 *)c->d_pop[0],
                                                                   (uint32_t)c->Nf, ps);
                    grid = gp;
                    break;
                }
                if (reduce)
                    k_sparse_even_h4<K, true><<<g4, 256, 0, c->stream>>>(
                        (__half *)c->d_pop[0], (uint32_t)c->Nf, ps, lds, red);
                else
                    k_sparse_even_h4<K, false><<<g4, 256, 0, c->stream>>>(
                        (__half *)c->d_pop[0], (uint32_t)c->Nf, ps, lds, red);
                grid = reduce ? groups : g4;
                break;
            }
        }
        if constexpr (sizeof(S) <= 4) {
            if (!odd && narrow_index(c)) {
                const unsigned g2 = (unsigned)((c->Nf + 511) / 512);
                if (reduce)
                    k_sparse_even_x2<S, K, true><<<g2, 256, 0, c->stream>>>(
                        (S *)c->d_pop[0], (uint32_t)c->Nf, p, lds, sts, red);
                else
                    k_sparse_even_x2<S, K, false><<<g2, 256, 0, c->stream>>>(
                        (S *)c->d_pop[0], (uint32_t)c->Nf, p, lds, sts, red);
                grid = reduce ? groups : g2;
                break;
            }
        }
        if (odd) {
            const unsigned tg = (unsigned)((c->Nf + 256 * LBM_SPARSE_ODD_NPT - 1) /
                                           (256 * LBM_SPARSE_ODD_NPT));
            const SparseMap sm = sparse_map(c);
            S *A = (S *)c->d_pop[0];
            const uint32_t Nf = (uint32_t)c->Nf;
            bool lean = false;
            if constexpr (sizeof(S) <= 4 && LBM_ODD_LEAN) {
                if (narrow_index(c) && c->d_orec) {
                    const OddMap o = odd_map(c);
                    switch (odd_nodes_per_thread<S, K>(c)) {
                    case 1: launch_odd_lean<S, 1, K>(c, reduce, o, A, Nf, p, lds, sts, red); break;
                    case 2: launch_odd_lean<S, 2, K>(c, reduce, o, A, Nf, p, lds, sts, red); break;
                    default: launch_odd_lean<S, 4, K>(c, reduce, o, A, Nf, p, lds, sts, red); break;
                    }
                    lean = true;
                }
            }
            if (lean) {
            } else if (narrow_index(c)) {
                if (reduce)
                    k_sparse_odd_t<S, uint32_t, LBM_SPARSE_ODD_NPT, K, true>
                        <<<tg, 256, 0, c->stream>>>(A, sm, Nf, p, lds, sts, red);
                else
                    k_sparse_odd_t<S, uint32_t, LBM_SPARSE_ODD_NPT, K, false>
                        <<<tg, 256, 0, c->stream>>>(A, sm, Nf, p, lds, sts, red);
            } else {
                if (reduce)
                    k_sparse_odd_t<S, size_t, LBM_SPARSE_ODD_NPT, K, true>
                        <<<tg, 256, 0, c->stream>>>(A, sm, Nf, p, lds, sts, red);
                else
                    k_sparse_odd_t<S, size_t, LBM_SPARSE_ODD_NPT, K, false>
                        <<<tg, 256, 0, c->stream>>>(A, sm, Nf, p, lds, sts, red);
            }
            grid = reduce ? groups : tg;
        } else if (narrow_index(c)) {  // even steps, FP64 storage
            k_sparse<S, false, uint32_t, K><<<grid, bs, 0, c->stream>>>(
                (S *)c->d_pop[0], sparse_map(c), (uint32_t)c->Nf, p, lds, sts, red);
        } else {
            k_sparse<S, false, size_t, K><<<grid, bs, 0, c->stream>>>(
                (S *)c->d_pop[0], sparse_map(c), (uint32_t)c->Nf, p, lds, sts, red);
        }
        break;
    }
    c->launches++;
    c->steps++;
    if (reduce) return (int)grid;
    return 0;
}

template <typename S>
int launch_step_t(lbm_ctx *c, bool reduce) {
    using Cm = typename Store<S>::C;
    const Collide<Cm> p = make_collide<Cm>(c->s, c->F, c->opt.linear_eq, c->opt.collision == 0);
    return p.trt ? launch_step_k<S, kCollideTrt>(c, reduce, p)
                 : launch_step_k<S, kCollideMrt>(c, reduce, p);
}

static StateView make_view(const lbm_ctx *c) {
    StateView v;
    v.layout = c->opt.layout;
    v.parity = (int)(c->steps & 1);
    v.units = (uint32_t)(c->opt.layout == LBM_LAYOUT_SPARSE ? c->Nf : c->N);
    v.lw = c->d_lw;
    v.sm = sparse_map(c);
    v.d = Dims{c->Lx, c->Ly, c->Lz, (uint32_t)c->N};
    return v;
}

static const void *cur_pop(const lbm_ctx *c) {
    return c->opt.layout == LBM_LAYOUT_AB ? c->d_pop[c->cur] : c->d_pop[0];
}

template <typename S>
int launch_velocity_t(lbm_ctx *c, double *u_dev, bool reduce) {
    StateView v = make_view(c);
    const int bs = 256;
    const unsigned grid = nblocks(v.units, bs);
    if (grid == 0) return 0;
    Reduce red{reduce ? c->d_partials : nullptr, c->d_flag};
    const float lds = c->fp16_scale > 0.f ? 1.0f / c->fp16_scale : 1.0f;
    if constexpr (sizeof(typename Store<S>::C) == 4) {
        if (!u_dev && reduce) {
            const float Fx = (float)c->F[0], Fy = (float)c->F[1], Fz = (float)c->F[2];
            if (v.layout == LBM_LAYOUT_SPARSE)
                k_velocity_sum<S, true><<<grid, bs, 0, c->stream>>>((const S *)cur_pop(c), v, Fx, Fy,
                                                                    Fz, lds, red);
            else
                k_velocity_sum<S, false><<<grid, bs, 0, c->stream>>>((const S *)cur_pop(c), v, Fx,
                                                                     Fy, Fz, lds, red);
            c->launches++;
            return (int)grid;
        }
    }
    k_velocity<S><<<grid, bs, 0, c->stream>>>((const S *)cur_pop(c), v, c->d_fidx, c->F[0], c->F[1],
                                              c->F[2], lds, u_dev, red);
    c->launches++;
    return (int)grid;
}

template <typename S>
void launch_export_t(lbm_ctx *c, double *f_dev) {
    StateView v = make_view(c);
    const unsigned grid = nblocks(v.units, 256);
    if (grid == 0) return;
    const float lds = c->fp16_scale > 0.f ? 1.0f / c->fp16_scale : 1.0f;
    k_export<S><<<grid, 256, 0, c->stream>>>((const S *)cur_pop(c), v, c->d_fidx, lds, f_dev);
    c->launches++;
}

template <typename S>
void launch_import_t(lbm_ctx *c, const double *f_dev) {
    StateView v = make_view(c);
    const unsigned grid = nblocks(v.units, 256);
    if (grid == 0) return;
    const float sts = c->fp16_scale > 0.f ? c->fp16_scale : 1.0f;
    // AB: the post-collision state is the current array
    k_import<S><<<grid, 256, 0, c->stream>>>((S *)cur_pop(c), v, c->d_fidx, sts, f_dev);
    c->launches++;
}

template <typename S>
void launch_export_at_t(lbm_ctx *c, const int64_t *nodes_dev, int count, double *f_dev) {
    StateView v = make_view(c);
    const float lds = c->fp16_scale > 0.f ? 1.0f / c->fp16_scale : 1.0f;
    k_export_at<S><<<nblocks(count, 256), 256, 0, c->stream>>>((const S *)cur_pop(c), v, c->d_fidx,
                                                               nodes_dev, count, lds, f_dev);
    c->launches++;
}

void launch_export_at(lbm_ctx *c, const int64_t *nodes_dev, int count, double *f_dev) {
    switch (c->opt.precision) {
    case LBM_FP64: launch_export_at_t<double>(c, nodes_dev, count, f_dev); break;
    case LBM_FP32_SHIFTED: launch_export_at_t<float>(c, nodes_dev, count, f_dev); break;
    default: launch_export_at_t<__half>(c, nodes_dev, count, f_dev); break;
    }
}

// Dispatch on the storage precision.
int launch_step(lbm_ctx *c, bool reduce) {
    switch (c->opt.precision) {
    case LBM_FP64: return launch_step_t<double>(c, reduce);
    case LBM_FP32_SHIFTED: return launch_step_t<float>(c, reduce);
    default: return launch_step_t<__half>(c, reduce);
    }
}

int launch_velocity(lbm_ctx *c, double *u_dev, bool reduce) {
    switch (c->opt.precision) {
    case LBM_FP64: return launch_velocity_t<double>(c, u_dev, reduce);
    case LBM_FP32_SHIFTED: return launch_velocity_t<float>(c, u_dev, reduce);
    default: return launch_velocity_t<__half>(c, u_dev, reduce);
    }
}

void launch_export(lbm_ctx *c, double *f_dev) {
    switch (c->opt.precision) {
    case LBM_FP64: launch_export_t<double>(c, f_dev); break;
    case LBM_FP32_SHIFTED: launch_export_t<float>(c, f_dev); break;
    default: launch_export_t<__half>(c, f_dev); break;
    }
}

void launch_import(lbm_ctx *c, const double *f_dev) {
    switch (c->opt.precision) {
    case LBM_FP64: launch_import_t<double>(c, f_dev); break;
    case LBM_FP32_SHIFTED: launch_import_t<float>(c, f_dev); break;
    default: launch_import_t<__half>(c, f_dev); break;
    }
}

void launch_finalize(lbm_ctx *c, int nblk, double inv_total, double *out_dev) {
    k_finalize<<<1, 1024, 0, c->stream>>>(c->d_partials, nblk, inv_total, out_dev);
    c->launches++;
}

}  // namespace lbm
