// Internal definitions shared by the CUDA translation units of liblbm_gb300.
// D3Q19 lattice constants, kernel parameter blocks, storage traits and the
// context structure behind the opaque lbm_ctx of include/lbm.h.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "lbm.h"

namespace lbm {

constexpr int Q = 19;

// D3Q19 velocities: rest, six axis links (+ before -), twelve edge links in
// opposite pairs.  The opposite of i is i+1 for odd i, i-1 for even i > 0.
__host__ __device__ constexpr int cx(int i) {
    return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13)
               ? 1
               : ((i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0);
}
__host__ __device__ constexpr int cy(int i) {
    return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17)
               ? 1
               : ((i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0);
}
__host__ __device__ constexpr int cz(int i) {
    return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18)
               ? 1
               : ((i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0);
}
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }

__host__ __device__ constexpr double weight(int i) {
    return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
}

// Bit 31 of a dense link word marks a solid voxel; bit i (1..18) marks a
// bounceback link: the upstream neighbour x - c_i is solid.
constexpr uint32_t SOLID_BIT = 1u << 31;
// Bit 30 marks a full-way bounceback voxel: a solid voxel with a fluid link
// neighbour that reflects what streams into it (full-way mode only; its
// other bits are 0, and so are the bounceback bits of fluid nodes there).
constexpr uint32_t BBNODE_BIT = 1u << 30;
constexpr uint32_t NOT_FLUID = SOLID_BIT | BBNODE_BIT;

// Relaxation rates and drive in the arithmetic type of the kernel.
template <typename T>
struct Collide {
    T se, seps, sq, snu, spi, sm;  // diag(S) of eq. (MRT params), grouped
    T he, heps, hq, hnu, hpi, hm;  // 1 - s/2 of each group (forcing weight)
    T Fx, Fy, Fz;                  // body force density
    T q;                           // weight of the quadratic equilibrium / forcing terms
    int linear;                    // drop quadratic equilibrium / forcing terms
    int trt;                       // one even and one odd rate: link-basis collision
};

// Collision parameters in the kernel's arithmetic type from the FP64 rates
// s[19] (moment order) and force.  Every kernel that steps a lattice takes
// its parameters from here, so all of them see the same values.
template <typename T>
inline Collide<T> make_collide(const double s[19], const double F[3], int linear,
                               int allow_trt = 1) {
    Collide<T> p;
    p.se = (T)s[1];
    p.seps = (T)s[2];
    p.sq = (T)s[4];
    p.snu = (T)s[9];
    p.spi = (T)s[10];
    p.sm = (T)s[16];
    p.he = (T)(1.0 - 0.5 * s[1]);
    p.heps = (T)(1.0 - 0.5 * s[2]);
    p.hq = (T)(1.0 - 0.5 * s[4]);
    p.hnu = (T)(1.0 - 0.5 * s[9]);
    p.hpi = (T)(1.0 - 0.5 * s[10]);
    p.hm = (T)(1.0 - 0.5 * s[16]);
    p.Fx = (T)F[0];
    p.Fy = (T)F[1];
    p.Fz = (T)F[2];
    p.q = linear ? T(0) : T(1);
    p.linear = linear;
    // s_e = s_eps = s_nu = s_pi and s_q = s_m: the link-basis TRT form applies
    p.trt = allow_trt && s[1] == s[9] && s[2] == s[9] && s[10] == s[9] && s[16] == s[4];
    return p;
}

// The collision of values scaled by sigma = 2^S: the FP16 storage kernels
// that collide the stored halves as they are (h = 2^S (f - w)), without the
// 2^-S multiply on load and the 2^S multiply on store.  The force is scaled
// by sigma and the weight of the quadratic terms by 1/sigma.  Every
// intermediate of the collision is then the unscaled one times an exact
// power of two (both collision forms are sums and products of the values,
// the force and constants, each product of two scaled factors met by q), so
// the halves stored are bitwise those of the scaled loads and stores, and
// the momentum is sigma times the unscaled one.
inline Collide<float> scaled_collide(Collide<float> p, float sigma) {
    p.Fx *= sigma;
    p.Fy *= sigma;
    p.Fz *= sigma;
    p.q /= sigma;
    return p;
}

struct Dims {
    int Lx, Ly, Lz;
    uint32_t N;  // Lx*Ly*Lz < 2^31
};

// Storage traits: S is the stored type, C the arithmetic type.
template <typename S>
struct Store;
template <>
struct Store<double> {
    using C = double;
    static __device__ __forceinline__ double ld(const double *p, float) { return *p; }
    static __device__ __forceinline__ void st(double *p, double v, float) { *p = v; }
};
template <>
struct Store<float> {
    using C = float;
    static __device__ __forceinline__ float ld(const float *p, float) { return *p; }
    static __device__ __forceinline__ void st(float *p, float v, float) { *p = v; }
};
template <>
struct Store<__half> {
    using C = float;
    // stored value h = 2^S (f - w); `scale` carries 2^S on store, 2^-S on load
    // (rounded multiplies: never fused into the arithmetic around them)
    static __device__ __forceinline__ float ld(const __half *p, float inv) {
        return __fmul_rn(__half2float(*p), inv);
    }
    static __device__ __forceinline__ void st(__half *p, float v, float sc) {
        *p = __float2half_rn(__fmul_rn(v, sc));
    }
};

// Sparse-layout row metadata, one entry per 32-voxel word of an x-row
// (row R = y + Ly*z): bit b of `bits` is set iff voxel x = 32w + b is fluid;
// `base` is the fluid index of the first fluid node at x >= 32w of the row
// (equivalently the number of fluid nodes before that position in node
// order).  The fluid index of a fluid voxel (x, R) is then
// base + popc(bits & ((1 << (x & 31)) - 1)).
struct __align__(8) RowWord {
    uint32_t bits;
    int32_t base;
};

// Everything the sparse kernels need to find upstream fluid indices.
// mLx, mLy: ceil(2^64 / L), so that floor(n / L) = umul64hi(n, m) for any
// n < 2^32 and L < 2^31 (the rounding error n (m - 2^64/L) / 2^64 stays below
// 2^-32, smaller than the distance 1/L of a non-integer n/L to the next
// integer).
struct SparseMap {
    const int32_t *fidx;
    const uint32_t *bb;
    const uint2 *nb;  // per fluid node {node index, bounceback bits}: one 8-byte load
    const RowWord *rw;
    const int32_t *rstart;
    int Lx, Ly, Lz, Wr;
    uint64_t mLx, mLy;
    int *flag;  // the context's device flag (bounds-check build: FLAG_BOUNDS)
};

// Bits of a context's device flag.
constexpr int FLAG_NONFINITE = 1;  // a non-finite density or momentum
constexpr int FLAG_BOUNDS = 2;     // an index out of range (bounds-check build)

// Bounds-check build (-DLBM_BOUNDS_CHECK): every computed offset into the
// population, index-record, row-word and row-start arrays is range-checked
// before the access; an offset out of range skips the access and raises
// FLAG_BOUNDS in the context's flag, which lbm_device_flags reports.  It
// never traps, so the context stays usable.  In the normal build in_range
// is the constant true and compiles away.
#ifdef LBM_BOUNDS_CHECK
constexpr bool kBoundsCheck = true;
#else
constexpr bool kBoundsCheck = false;
#endif
__device__ __forceinline__ bool in_range(uint64_t i, uint64_t n, int *flag) {
    if (!kBoundsCheck) return true;
    if (i < n) return true;
    if (flag) atomicOr(flag, FLAG_BOUNDS);
    return false;
}
// p[i], or 0 where i >= n (bounds-check build only; plain p[i] otherwise).
template <typename T>
__device__ __forceinline__ T load_chk(const T *p, uint64_t i, uint64_t n, int *flag) {
    return in_range(i, n, flag) ? p[i] : T{};
}

// The odd AA step of the sparse layout with its index arithmetic cut down
// (k_sparse_odd_l).  Set up once per context:
//  rec[k]  {padded row p, bounceback bits | x << 19} of fluid node k, where
//          p = (y + 1) + (Ly + 2)(z + 1) numbers the rows of the lattice
//          padded by one ghost row on each side in y and z (needs Lx < 2^13);
//  rwp     the row words (RowWord) of the padded rows, Wr per row, the ghost
//          rows copies of the rows they stand for (periodic in y and z);
//  rse     per padded row {fluid index of the row's first fluid voxel, one
//          past its last}.
// Neighbour row slot s of padded row p is p + dy_s + (Ly + 2) dz_s, so each
// slot's base pointer is offset once on the host (rws, rse) and a node's
// row word w of slot s is rws[s][p Wr + w]: no division, no wrap test.
// slot[j] = j Nf puts the slot offsets in the kernel's parameter bank.
struct OddMap {
    const uint2 *rec;
    const RowWord *rws[8];  // rwp shifted to neighbour row slot s
    const int2 *rse[9];     // rse shifted to slot s; [8]: the own row
    uint32_t slot[19];      // j * Nf
    uint32_t Wr, Lx;
    // bounds-check build: the unshifted tables and their sizes
    const RowWord *rwp;
    const int2 *rse0;
    int32_t roff[9];        // row offset of each slot (0 for the own row)
    uint32_t nprows;        // padded rows
    int *flag;
};
constexpr uint32_t kOddMaxLx = 1u << 13;  // x must fit 13 bits of the record

__host__ __forceinline__ uint64_t div_magic(uint32_t L) {
    // ceil(2^64 / L) for L >= 2; L == 1 is handled by the caller
    return L <= 1 ? 0 : (~uint64_t(0)) / L + 1;
}

__device__ __forceinline__ uint32_t fast_div(uint32_t n, uint32_t L, uint64_t m) {
    return L == 1 ? n : (uint32_t)__umul64hi((uint64_t)n, m);
}

// Population access that bypasses L1 (cached in L2 only): needed where one
// kernel launch reads, in a later step, what other blocks wrote in an
// earlier one (the persistent batch kernel), since L1 is not coherent
// across SMs and is only invalidated between launches.
template <typename S>
struct StoreL2 {
    using C = typename Store<S>::C;
    static __device__ __forceinline__ C ld(const S *p, float s);
    static __device__ __forceinline__ void st(S *p, C v, float s);
};
template <>
__device__ __forceinline__ double StoreL2<double>::ld(const double *p, float) { return __ldcg(p); }
template <>
__device__ __forceinline__ void StoreL2<double>::st(double *p, double v, float) { __stcg(p, v); }
template <>
__device__ __forceinline__ float StoreL2<float>::ld(const float *p, float) { return __ldcg(p); }
template <>
__device__ __forceinline__ void StoreL2<float>::st(float *p, float v, float) { __stcg(p, v); }
template <>
__device__ __forceinline__ float StoreL2<__half>::ld(const __half *p, float inv) {
    const unsigned short b = __ldcg(reinterpret_cast<const unsigned short *>(p));
    return __fmul_rn(__half2float(__ushort_as_half(b)), inv);
}
template <>
__device__ __forceinline__ void StoreL2<__half>::st(__half *p, float v, float sc) {
    __stcg(reinterpret_cast<unsigned short *>(p), __half_as_ushort(__float2half_rn(__fmul_rn(v, sc))));
}

// Per-launch reduction target: per-block partial sums of (ux, uy, uz) in
// double, and a device flag raised on non-finite density or momentum.
struct Reduce {
    double *partials;  // [gridDim.x][3], or nullptr for no reduction
    int *flag;
};

int launch_error(cudaError_t e);

// A named NVTX range over a host scope (convergence chunks, batch chunks,
// adjoint iterations), visible in profilers' timelines; no cost without one.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

}  // namespace lbm

// The host-side context (device pointers, options, counters).
#include "lbm_ctx.h"

