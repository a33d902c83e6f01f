// Upstream fluid indices of the sparse layout, computed instead of stored.
//
// Fluid nodes are numbered in node order (x fastest), so along an x-row the
// fluid indices of consecutive fluid voxels are consecutive.  For the 8
// neighbouring rows (y +- 1, z +- 1) a node needs the fluid index at its own
// x: the row's RowWord for x's 32-voxel word gives it as
// base + popc(bits below x).  The neighbours at x - 1 and x + 1 of a row then
// follow by -1 / +fluid(x), with the periodic wrap in x taken from the row
// start table.  The per-node bounceback bits say which upstream voxels are
// solid, so only fluid upstream indices are ever formed.  Row metadata is
// N/4 bytes in total and is re-read by the nine rows around it within a few
// microseconds, so it is served from L1/L2; per fluid node an odd step streams
// only its node index and bounceback bits (8 bytes) instead of an 18-entry
// neighbour table (72 bytes).
#pragma once

#include "lbm_internal.cuh"

namespace lbm {

// Neighbour-row slot of direction j (rows by (dy, dz) = (-cy, -cz)):
// 0 (-1,0)  1 (+1,0)  2 (0,-1)  3 (0,+1)  4 (-1,-1)  5 (+1,+1)  6 (-1,+1)  7 (+1,-1)
__host__ __device__ constexpr int row_slot(int j) {
    return (cy(j) == 1 && cz(j) == 0)     ? 0
           : (cy(j) == -1 && cz(j) == 0)  ? 1
           : (cy(j) == 0 && cz(j) == 1)   ? 2
           : (cy(j) == 0 && cz(j) == -1)  ? 3
           : (cy(j) == 1 && cz(j) == 1)   ? 4
           : (cy(j) == -1 && cz(j) == -1) ? 5
           : (cy(j) == 1 && cz(j) == -1)  ? 6
           : (cy(j) == -1 && cz(j) == 1)  ? 7
                                          : -1;
}
// Direction with cx = 0 whose upstream voxel is (x, row of slot s).
__host__ __device__ constexpr int slot_axis_dir(int s) {
    return s == 0 ? 3 : s == 1 ? 4 : s == 2 ? 5 : s == 3 ? 6 : s == 4 ? 15 : s == 5 ? 16
                                                        : s == 6 ? 17 : 18;
}
__host__ __device__ constexpr int slot_dy(int s) {
    return (s == 0 || s == 4 || s == 6) ? -1 : (s == 1 || s == 5 || s == 7) ? 1 : 0;
}
__host__ __device__ constexpr int slot_dz(int s) {
    return (s == 2 || s == 4 || s == 7) ? -1 : (s == 3 || s == 5 || s == 6) ? 1 : 0;
}
// Bounceback bits of all directions reading row slot s.
__host__ __device__ constexpr uint32_t slot_dirs(int s) {
    uint32_t m = 0;
    for (int j = 1; j < Q; ++j)
        if (row_slot(j) == s) m |= 1u << j;
    return m;
}

struct SparseNode {
    uint32_t k, bits;
    int x, y, z;
    bool xlo, xhi;    // x == 0, x == Lx - 1: the x-neighbour wraps around the row
    int32_t rank[8];  // fluid index of the first fluid voxel at >= x in each neighbour row

    __device__ __forceinline__ void init(uint32_t kk, const SparseMap &m) {
        const uint2 v = __ldg(m.nb + kk);
        init_from(kk, v.x, v.y, m);
    }

    // One row word and one row-start entry (bounds-check build: range-checked).
    __device__ __forceinline__ uint2 row_word(const SparseMap &m, uint32_t at) const {
        if (!in_range(at, (uint64_t)m.Ly * m.Lz * m.Wr, m.flag)) return make_uint2(0u, 0u);
        return __ldg(reinterpret_cast<const uint2 *>(m.rw) + at);
    }
    __device__ __forceinline__ int32_t row_start(const SparseMap &m, uint32_t at) const {
        if (!in_range(at, (uint64_t)m.Ly * m.Lz + 1, m.flag)) return 0;
        return __ldg(m.rstart + at);
    }

    // n: node index of fluid node kk, b: its bounceback bits
    __device__ __forceinline__ void init_from(uint32_t kk, uint32_t n, uint32_t b,
                                              const SparseMap &m) {
        k = kk;
        bits = b;
        const uint32_t R = fast_div(n, (uint32_t)m.Lx, m.mLx);
        x = (int)(n - R * (uint32_t)m.Lx);
        z = (int)fast_div(R, (uint32_t)m.Ly, m.mLy);
        y = (int)(R - (uint32_t)z * (uint32_t)m.Ly);
        xlo = x == 0;
        xhi = x == m.Lx - 1;
        // word offsets of the rows y-1, y, y+1 and planes z-1, z, z+1
        const uint32_t LyWr = (uint32_t)m.Ly * (uint32_t)m.Wr;
        const uint32_t yo[3] = {(uint32_t)(y == 0 ? m.Ly - 1 : y - 1) * m.Wr, (uint32_t)y * m.Wr,
                                (uint32_t)(y == m.Ly - 1 ? 0 : y + 1) * m.Wr};
        const uint32_t zo[3] = {(uint32_t)(z == 0 ? m.Lz - 1 : z - 1) * LyWr, (uint32_t)z * LyWr,
                                (uint32_t)(z == m.Lz - 1 ? 0 : z + 1) * LyWr};
        const uint32_t w = (uint32_t)x >> 5;
        const uint32_t below = (1u << (x & 31)) - 1u;
        // all eight rows, also where every upstream voxel in a row is solid
        // (unused then): issuing the loads unconditionally measured faster
        // than branching on the bounceback bits
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            const uint2 rw = row_word(m, yo[1 + slot_dy(s)] + zo[1 + slot_dz(s)] + w);
            rank[s] = (int32_t)rw.y + __popc(rw.x & below);
        }
    }

    // row index of neighbour slot s (periodic in y and z)
    __device__ __forceinline__ uint32_t nrow(const SparseMap &m, int s) const {
        int yy = y + slot_dy(s), zz = z + slot_dz(s);
        yy = yy < 0 ? yy + m.Ly : (yy >= m.Ly ? yy - m.Ly : yy);
        zz = zz < 0 ? zz + m.Lz : (zz >= m.Lz ? zz - m.Lz : zz);
        return (uint32_t)yy + (uint32_t)m.Ly * (uint32_t)zz;
    }

    // up() for a node with 0 < x < Lx - 1 (no periodic wrap in x).
    __device__ __forceinline__ uint32_t up_interior(int j) const {
        if (j == 0) return k;
        const int dx = cx(j);
        if (cy(j) == 0 && cz(j) == 0) return dx > 0 ? k - 1 : k + 1;
        const int s = row_slot(j);
        if (dx == 0) return (uint32_t)rank[s];
        if (dx > 0) return (uint32_t)(rank[s] - 1);
        return (uint32_t)rank[s] + ((bits >> slot_axis_dir(s)) & 1u ? 0u : 1u);
    }

    // Fluid index of the upstream voxel x - c_j; valid only where bit j of
    // the bounceback bits is clear (the upstream voxel is fluid).
    __device__ __forceinline__ uint32_t up(int j, const SparseMap &m) const {
        if (j == 0) return k;
        const int dx = cx(j);
        if (cy(j) == 0 && cz(j) == 0) {  // own row
            if (dx > 0) {
                if (xlo) return (uint32_t)(row_start(m, (uint32_t)y + (uint32_t)m.Ly * z + 1) - 1);
                return k - 1;
            }
            if (xhi) return (uint32_t)row_start(m, (uint32_t)y + (uint32_t)m.Ly * z);
            return k + 1;
        }
        const int s = row_slot(j);
        if (dx == 0) return (uint32_t)rank[s];
        if (dx > 0) {  // upstream at x - 1
            if (xlo) return (uint32_t)(row_start(m, nrow(m, s) + 1) - 1);
            return (uint32_t)(rank[s] - 1);
        }
        // upstream at x + 1: skip (x, row) if that voxel is fluid
        if (xhi) return (uint32_t)row_start(m, nrow(m, s));
        return (uint32_t)rank[s] + ((bits >> slot_axis_dir(s)) & 1u ? 0u : 1u);
    }
};

}  // namespace lbm
