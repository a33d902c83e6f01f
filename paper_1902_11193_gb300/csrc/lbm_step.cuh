// One in-place (AA pattern) stream-collide update of one unit, shared by the
// single-lattice kernels (lbm_kernels.cu) and the batched persistent kernel
// (lbm_batch.cu), so both run the same arithmetic on the same locations.
//
// Even step: the 19 populations are read from the node's own slots j and the
// post-collision value of direction opp(j) is written back to slot j.  Odd
// step: population j is read from slot opp(j) of the upstream neighbour
// x - c_j (slot j of the node itself when that neighbour is solid: halfway
// bounceback) and the post-collision value of opp(j) is written back to that
// same place.
#pragma once

#include "lbm_collide.cuh"
#include "lbm_sparse.cuh"

namespace lbm {

// Sum of the momenta (jx, jy, jz) of a block's units, one unit per thread,
// written by threads 0..2 to out[0..2]; raises bit 0 of *flag (if given) on
// a non-finite momentum.  Every thread of the block calls it (it synchronises
// the block).  The order is fixed, so the result is reproducible, and the
// single-lattice and batched kernels share it, so they agree bit for bit.
//
// FP64 arithmetic is scarce on this GPU (a shuffle tree in FP64 cost about
// 1.3 ms per 5e7 units), so FP32 momenta are summed per warp in FP32 with
// the exact error of every addition carried along (Knuth's two-sum): the
// warp's sum hi + lo is off by at most about 2^-43 of the sum of the
// magnitudes (the 31 carried errors are themselves added in FP32).  Only the warp sums and the
// block total are formed in FP64.  FP64 momenta use the same tree in FP64.
__device__ __forceinline__ void two_sum_step(float &s, float &e, int o) {
    const float ts = __shfl_down_sync(0xffffffffu, s, o);
    const float te = __shfl_down_sync(0xffffffffu, e, o);
    const float x = __fadd_rn(s, ts);
    const float z = __fsub_rn(x, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(x, z)), __fsub_rn(ts, z));
    e = __fadd_rn(__fadd_rn(e, te), err);
    s = x;
}

template <typename C>
__device__ __forceinline__ double warp_momentum_sum(C v) {
    if constexpr (sizeof(C) == 8) {
        double d = v;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
        return d;
    } else {
        float s = v, e = 0.0f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) two_sum_step(s, e, o);
        return (double)s + (double)e;
    }
}

// The two halves of block_momentum_sum, for kernels that reduce several
// groups per block with one synchronisation: the warp sums of a group go to
// sm[warp][0..2] (lane 0 writes); after a __syncthreads, thread a (< 3) of
// any warp adds the group's warps in order.  Same arithmetic, same order.
template <typename C>
__device__ __forceinline__ void warp_momentum_store(C jx, C jy, C jz, bool fluid,
                                                    double (*sm)[3], int *flag) {
    if (flag && fluid && !(isfinite(jx) && isfinite(jy) && isfinite(jz))) atomicOr(flag, 1);
    const C zero = C(0);
    const double w0 = warp_momentum_sum<C>(fluid ? jx : zero);
    const double w1 = warp_momentum_sum<C>(fluid ? jy : zero);
    const double w2 = warp_momentum_sum<C>(fluid ? jz : zero);
    if ((threadIdx.x & 31) == 0) {
        sm[threadIdx.x >> 5][0] = w0;
        sm[threadIdx.x >> 5][1] = w1;
        sm[threadIdx.x >> 5][2] = w2;
    }
}

__device__ __forceinline__ double group_momentum_total(const double (*sm)[3], int a) {
    double acc = 0.0;
    const int nw = (int)(blockDim.x >> 5);
    for (int i = 0; i < nw; ++i) acc += sm[i][a];
    return acc;
}

template <typename C>
__device__ __forceinline__ void block_momentum_sum(C jx, C jy, C jz, bool fluid, double *out,
                                                   int *flag) {
    if (flag && fluid && !(isfinite(jx) && isfinite(jy) && isfinite(jz))) atomicOr(flag, 1);
    const C zero = C(0);
    const double w[3] = {warp_momentum_sum<C>(fluid ? jx : zero),
                         warp_momentum_sum<C>(fluid ? jy : zero),
                         warp_momentum_sum<C>(fluid ? jz : zero)};
    __shared__ double sm[32][3];
    if ((threadIdx.x & 31) == 0) {
        sm[threadIdx.x >> 5][0] = w[0];
        sm[threadIdx.x >> 5][1] = w[1];
        sm[threadIdx.x >> 5][2] = w[2];
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double acc = 0.0;
        const int nw = (int)(blockDim.x >> 5);
        for (int i = 0; i < nw; ++i) acc += sm[i][threadIdx.x];
        out[threadIdx.x] = acc;
    }
    __syncthreads();
}

struct DenseNode {
    int x, xm, xp;
    uint32_t row[3][3];  // Lx*(y' + Ly*z') for y' in {y-1, y, y+1}, z' likewise (wrapped)

    __device__ __forceinline__ void init(uint32_t n, const Dims &d) {
        uint32_t t = n / (uint32_t)d.Lx;
        x = (int)(n - t * (uint32_t)d.Lx);
        int z = (int)(t / (uint32_t)d.Ly);
        int y = (int)(t - (uint32_t)z * (uint32_t)d.Ly);
        xm = x == 0 ? d.Lx - 1 : x - 1;
        xp = x == d.Lx - 1 ? 0 : x + 1;
        int ys[3] = {y == 0 ? d.Ly - 1 : y - 1, y, y == d.Ly - 1 ? 0 : y + 1};
        int zs[3] = {z == 0 ? d.Lz - 1 : z - 1, z, z == d.Lz - 1 ? 0 : z + 1};
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b)
                row[a][b] = (uint32_t)d.Lx * ((uint32_t)ys[a] + (uint32_t)d.Ly * (uint32_t)zs[b]);
    }
    // node index of the upstream neighbour x - c_j
    __device__ __forceinline__ uint32_t up(int j) const {
        int xs = cx(j) > 0 ? xm : (cx(j) < 0 ? xp : x);
        return (uint32_t)xs + row[1 - cy(j)][1 - cz(j)];
    }
};

// Location (flat offset) of logical direction j for node n of a dense AA lattice.
template <bool ODD>
__device__ __forceinline__ size_t aa_loc_dense(int j, uint32_t n, uint32_t w,
                                               const DenseNode &nd, uint32_t N) {
    if (!ODD || j == 0 || (w & (1u << j))) return (size_t)j * N + n;
    return (size_t)opp(j) * N + nd.up(j);
}

// Dense AA update of node n (link word w); returns false for solid nodes.
template <typename S, bool ODD, typename Acc = Store<S>, int K = kCollideRuntime>
__device__ __forceinline__ bool aa_dense_update(S *A, uint32_t n, uint32_t w, const Dims &d,
                                                const Collide<typename Store<S>::C> &p,
                                                float ld_scale, float st_scale,
                                                typename Store<S>::C &jx, typename Store<S>::C &jy,
                                                typename Store<S>::C &jz, int *flag = nullptr) {
    using C = typename Store<S>::C;
    if (w & SOLID_BIT) return false;
    DenseNode nd;
    if (ODD) nd.init(n, d);
    const uint64_t lim = (uint64_t)Q * d.N;
    C g[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        const size_t at = aa_loc_dense<ODD>(j, n, w, nd, d.N);
        g[j] = in_range(at, lim, flag) ? Acc::ld(A + at, ld_scale) : C(0);
    }
    collide_as<K, C>(g, p, jx, jy, jz);
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        const size_t at = aa_loc_dense<ODD>(j, n, w, nd, d.N);
        if (in_range(at, lim, flag)) Acc::st(A + at, g[opp(j)], st_scale);
    }
    return true;
}

// Locations (flat offsets into the population array) that an odd AA step
// of the sparse layout reads and writes for fluid node k, whose
// {node index, bounceback bits} record is `nb`: slot opp(j) of the upstream
// fluid node x - c_j, or slot j of k itself where that voxel is solid
// (halfway bounceback); loc[0] = k.
// Interior formulas for every node, then the periodic wrap in x for the few
// nodes on the x faces; measured faster than one path that tests for the
// wrap in every direction.
template <typename Idx>
__device__ __forceinline__ void odd_locations_of(const SparseNode &sn, const SparseMap &m,
                                                 uint32_t Nf, Idx loc[Q]) {
    const uint32_t k = sn.k;
    loc[0] = k;
#pragma unroll
    for (int j = 1; j < Q; ++j)
        loc[j] = (sn.bits & (1u << j)) ? (Idx)j * Nf + k : (Idx)opp(j) * Nf + sn.up_interior(j);
    if (sn.xlo || sn.xhi) {
#pragma unroll
        for (int j = 1; j < Q; ++j)
            if (cx(j) != 0 && !(sn.bits & (1u << j))) loc[j] = (Idx)opp(j) * Nf + sn.up(j, m);
    }
}

template <typename Idx>
__device__ __forceinline__ void odd_sparse_locations(const SparseMap &m, uint32_t Nf, uint32_t k,
                                                     uint2 nb, Idx loc[Q]) {
    SparseNode sn;
    sn.init_from(k, nb.x, nb.y, m);
    odd_locations_of<Idx>(sn, m, Nf, loc);
}

// odd_sparse_locations from an OddMap record: the same locations, bit for
// bit, with less index arithmetic (see OddMap).
__device__ __forceinline__ void odd_lean_locations(const OddMap &o, uint32_t k, uint2 rec,
                                                   uint32_t loc[Q]) {
    const uint32_t p = rec.x, bits = rec.y & 0x7FFFEu, x = rec.y >> 19;
    const uint32_t e = p * o.Wr + (x >> 5);
    const uint32_t below = (1u << (x & 31u)) - 1u;
    int32_t rank[8];
#pragma unroll
    for (int s = 0; s < 8; ++s) {
        uint2 v = make_uint2(0u, 0u);
        if (!kBoundsCheck || in_range((uint64_t)((int64_t)e + (int64_t)o.roff[s] * o.Wr),
                                      (uint64_t)o.nprows * o.Wr, o.flag))
            v = __ldg(reinterpret_cast<const uint2 *>(o.rws[s]) + e);
        rank[s] = (int32_t)v.y + __popc(v.x & below);
    }
    loc[0] = k;
#pragma unroll
    for (int j = 1; j < Q; ++j) {
        if (bits & (1u << j)) {
            loc[j] = o.slot[j] + k;
            continue;
        }
        const int dx = cx(j);
        uint32_t up;
        if (cy(j) == 0 && cz(j) == 0) {
            up = dx > 0 ? k - 1u : k + 1u;
        } else {
            const int s = row_slot(j);
            up = dx == 0  ? (uint32_t)rank[s]
                 : dx > 0 ? (uint32_t)(rank[s] - 1)
                          : (uint32_t)rank[s] + ((bits >> slot_axis_dir(s)) & 1u ? 0u : 1u);
        }
        loc[j] = o.slot[opp(j)] + up;
    }
    if (x == 0u || x == o.Lx - 1u) {  // the periodic wrap in x, from the row ends
#pragma unroll
        for (int j = 1; j < Q; ++j) {
            const int dx = cx(j);
            if (dx == 0 || (bits & (1u << j))) continue;
            if ((dx > 0 && x != 0u) || (dx < 0 && x != o.Lx - 1u)) continue;
            const int s = (cy(j) == 0 && cz(j) == 0) ? 8 : row_slot(j);
            int2 r = make_int2(0, 0);
            if (!kBoundsCheck ||
                in_range((uint64_t)((int64_t)p + o.roff[s]), (uint64_t)o.nprows, o.flag))
                r = __ldg(o.rse[s] + p);
            // upstream x - 1 of x = 0 is the row's last voxel; x + 1 of
            // x = Lx - 1 its first
            loc[j] = o.slot[opp(j)] + (dx > 0 ? (uint32_t)(r.y - 1) : (uint32_t)r.x);
        }
    }
}

// Gathers the 19 populations of one fluid node from `loc`, collides them
// and stores the post-collision values of the opposite directions back to
// the same locations (the AA pattern).
template <typename S, typename Idx, typename Acc = Store<S>, int K = kCollideRuntime>
__device__ __forceinline__ void aa_sparse_update_at(S *A, const SparseMap &m, uint32_t Nf,
                                                    const Idx loc[Q],
                                                    const Collide<typename Store<S>::C> &p,
                                                    float ld_scale, float st_scale,
                                                    typename Store<S>::C &jx,
                                                    typename Store<S>::C &jy,
                                                    typename Store<S>::C &jz) {
    using C = typename Store<S>::C;
    const uint64_t lim = (uint64_t)Q * Nf;
    C g[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j)
        g[j] = in_range(loc[j], lim, m.flag) ? Acc::ld(A + loc[j], ld_scale) : C(0);
    collide_as<K, C>(g, p, jx, jy, jz);
#pragma unroll
    for (int j = 0; j < Q; ++j)
        if (in_range(loc[j], lim, m.flag)) Acc::st(A + loc[j], g[opp(j)], st_scale);
}

// Sparse AA update of fluid node k; an odd step takes the node's
// {node index, bounceback bits} as `nb` (already loaded).
template <typename S, bool ODD, typename Idx, typename Acc = Store<S>, int K = kCollideRuntime>
__device__ __forceinline__ void aa_sparse_update(S *A, const SparseMap &m, uint32_t Nf, uint32_t k,
                                                 uint2 nb, const Collide<typename Store<S>::C> &p,
                                                 float ld_scale, float st_scale,
                                                 typename Store<S>::C &jx,
                                                 typename Store<S>::C &jy,
                                                 typename Store<S>::C &jz) {
    Idx loc[Q];
    if (ODD) {
        odd_sparse_locations<Idx>(m, Nf, k, nb, loc);
    } else {
#pragma unroll
        for (int j = 0; j < Q; ++j) loc[j] = (Idx)j * Nf + k;
    }
    aa_sparse_update_at<S, Idx, Acc, K>(A, m, Nf, loc, p, ld_scale, st_scale, jx, jy, jz);
}

}  // namespace lbm
