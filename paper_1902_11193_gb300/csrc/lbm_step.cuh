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
                                                typename Store<S>::C &jz) {
    using C = typename Store<S>::C;
    if (w & SOLID_BIT) return false;
    DenseNode nd;
    if (ODD) nd.init(n, d);
    C g[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) g[j] = Acc::ld(A + aa_loc_dense<ODD>(j, n, w, nd, d.N), ld_scale);
    collide_as<K, C>(g, p, jx, jy, jz);
#pragma unroll
    for (int j = 0; j < Q; ++j)
        Acc::st(A + aa_loc_dense<ODD>(j, n, w, nd, d.N), g[opp(j)], st_scale);
    return true;
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
    using C = typename Store<S>::C;
    Idx loc[Q];
    if (ODD) {
        SparseNode sn;
        sn.init_from(k, nb.x, nb.y, m);
        loc[0] = k;
        // Interior formulas for every node, then the periodic wrap in x for
        // the few nodes on the x faces; measured faster than one path that
        // tests for the wrap in every direction.
#pragma unroll
        for (int j = 1; j < Q; ++j)
            loc[j] = (sn.bits & (1u << j)) ? (Idx)j * Nf + k
                                            : (Idx)opp(j) * Nf + sn.up_interior(j);
        if (sn.xlo || sn.xhi) {
#pragma unroll
            for (int j = 1; j < Q; ++j)
                if (cx(j) != 0 && !(sn.bits & (1u << j))) loc[j] = (Idx)opp(j) * Nf + sn.up(j, m);
        }
    } else {
#pragma unroll
        for (int j = 0; j < Q; ++j) loc[j] = (Idx)j * Nf + k;
    }
    C g[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) g[j] = Acc::ld(A + loc[j], ld_scale);
    collide_as<K, C>(g, p, jx, jy, jz);
#pragma unroll
    for (int j = 0; j < Q; ++j) Acc::st(A + loc[j], g[opp(j)], st_scale);
}

}  // namespace lbm
