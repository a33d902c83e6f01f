// Steady fixed-point adjoint of the permeability (no counterpart in the
// paper's method; it differentiates the converged k of eq. perm_calc with
// respect to tau, the magic parameters and the body force).
//
// In the streamed variable h = S f* one time step is h -> S C(h).  At the
// steady state the adjoint psi of J = k along the drive d solves
//     psi = J_C(h)^T S^T psi + dJ/dh,      dJ/dh_i = nu c_{i,d} / (F_d N),
// and dk/dtheta = dJ/dtheta + (S^T psi) . dC/dtheta.
//  S^T     transposed streaming: the post-collision population i of x went
//          to x + c_i, or, where that voxel is solid, back into slot opp(i)
//          of x (the reversed bounceback link).
//  J_C^T   with C = M^-1 [m - S (m - m^eq) + (I - S/2) m^F], M^-1 = M^T D^-1:
//          J_C^T phi = M^T A^T D^-1 M phi with
//          A = I - S + S dm^eq/dm + (I - S/2) dm^F/dm.  m^eq and m^F depend on
//          m only through rho and j, so A^T relaxes every non-conserved moment
//          by (1 - s_k) and adds to the rho and j rows the sums over the
//          moments' equilibrium and forcing derivatives.
// The iteration converges at the rate of the forward problem.  Halfway
// bounceback in gaps one or two voxels wide gives both the forward step and
// this iteration modes of eigenvalue near -1, so the linearisation point is
// the mean of two consecutive streamed states, the residual compares
// iterates two apart (||psi_{n+1} - psi_{n-1}|| / ||psi_{n+1}||, reduced in
// FP64 every K steps) and the gradient uses the mean of the last two iterates.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "lbm_step.cuh"

#ifndef LBM_ADJ_LEAN
#define LBM_ADJ_LEAN 1  // 0: the FP32 sparse adjoint through the general index path
#endif

namespace lbm {

// Same unit machinery as the state readers (lbm_kernels.cu).
struct AdjView {
    int layout;
    uint32_t units;
    const uint32_t *lw;
    SparseMap sm;
    Dims d;
    OddMap om;  // sparse, Lx < 2^13: the odd step's lean index tables (om.rec null otherwise)
    // bounds-check build: a location outside the 19 * units slots
    __device__ __forceinline__ bool ok(size_t at) const { return in_range(at, (uint64_t)Q * units, sm.flag); }
};

struct AdjUnit {
    DenseNode d;
    SparseNode s;
    uint32_t bits;  // bit j: x - c_j is solid
    bool fluid;
    __device__ __forceinline__ void init(uint32_t u, const AdjView &v) {
        if (v.layout == LBM_LAYOUT_SPARSE) {
            s.init(u, v.sm);
            bits = s.bits;
            fluid = true;
        } else {
            bits = v.lw[u];
            fluid = !(bits & NOT_FLUID);
            if (fluid) d.init(u, v.d);
        }
    }
    // unit index of the upstream voxel x - c_j (valid where bit j is clear)
    __device__ __forceinline__ uint32_t up(int j, uint32_t u, const AdjView &v) const {
        return v.layout == LBM_LAYOUT_SPARSE ? s.up(j, v.sm) : d.up(j);
    }
};

// Where the streamed population i of unit u is kept by the current state
// (the same rule as the forward readers; duplicated here so the adjoint
// translation unit stands alone).
struct AdjState {
    int layout, parity;
};

__device__ __forceinline__ size_t streamed_loc(const AdjState &st, const AdjView &v, uint32_t u,
                                               int j, const AdjUnit &un) {
    if (st.layout == LBM_LAYOUT_AB) {
        if (j == 0) return u;
        if (un.bits & (1u << j)) return (size_t)opp(j) * v.units + u;
        return (size_t)j * v.units + un.up(j, u, v);
    }
    if (st.parity == 0 || j == 0 || (un.bits & (1u << j))) return (size_t)j * v.units + u;
    return (size_t)opp(j) * v.units + un.up(j, u, v);
}

// Block sums of NV values per thread into partials[NV blockIdx.x ..]: the
// warp sums of the momentum reduction (compensated FP32 for FP32, FP64 for
// FP64), then FP64 over the warps in order.
// ADD: add the block's sums into partials instead of storing them (one
// accumulator per block across the launches of a sweep).
template <typename T, int NV, bool ADD = false>
__device__ __forceinline__ void block_sum_n(const T x[NV], double *partials) {
    __shared__ double sm[32][NV];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int a = 0; a < NV; ++a) {
        const double w = warp_momentum_sum<T>(x[a]);
        if (lane == 0) sm[wid][a] = w;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double acc = 0.0;
        const int nw = (blockDim.x + 31) >> 5;
        for (int w = 0; w < nw; ++w) acc += sm[w][threadIdx.x];
        double &out = partials[(size_t)NV * blockIdx.x + threadIdx.x];
        out = ADD ? out + acc : acc;
    }
}

// Block sums of (a, b) into partials[2 blockIdx.x ..]: the warp sums of the
// momentum reduction (compensated FP32 for FP32, FP64 for FP64), then FP64.
// The residual of the adjoint iteration only steers when to stop, so its
// per-node terms are formed in the iteration's own precision; the FP64 form
// (76 FP64 operations per node) made a checking launch eleven times as long
// as a plain one on this GPU.
template <typename T>
__device__ __forceinline__ void block_sum2(T a, T b, double *partials) {
    const double wa = warp_momentum_sum<T>(a), wb = warp_momentum_sum<T>(b);
    __shared__ double sm[32][2];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        sm[wid][0] = wa;
        sm[wid][1] = wb;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double acc = 0.0;
        const int nw = (blockDim.x + 31) >> 5;
        for (int w = 0; w < nw; ++w) acc += sm[w][threadIdx.x];
        partials[2 * (size_t)blockIdx.x + threadIdx.x] = acc;
    }
}

// Sum_k w_k dP_k/dv_a over the moments whose equilibrium (v = j), forcing
// (v = F for d/du, v = u for d/dF) depends quadratically on the drive:
// the derivative of (38 v.X, -11 v.X, 2(2 vx Xx - vy Xy - vz Xz), -m9/2,
// 2(vy Xy - vz Xz), -m11/2, vx Xy + vy Xx, vy Xz + vz Xy, vx Xz + vz Xx)
// with respect to X_a, contracted with w.
template <typename T>
__device__ __forceinline__ T dotP(int a, T vx, T vy, T vz, const T w[Q]) {
    if (a == 0)
        return T(38) * vx * w[1] - T(11) * vx * w[2] + T(4) * vx * w[9] - T(2) * vx * w[10] +
               vy * w[13] + vz * w[15];
    if (a == 1)
        return T(38) * vy * w[1] - T(11) * vy * w[2] - T(2) * vy * w[9] + vy * w[10] +
               T(2) * vy * w[11] - vy * w[12] + vx * w[13] + vz * w[14];
    return T(38) * vz * w[1] - T(11) * vz * w[2] - T(2) * vz * w[9] + vz * w[10] -
           T(2) * vz * w[11] + vz * w[12] + vy * w[14] + vx * w[15];
}

// phi: the transposed-streamed adjoint at one node; h: the steady streamed
// populations there.  Returns b = D^-1 M phi and the shifted momentum of h.
// Shifted momentum j = sum_i c_i h_i + F/2 of a streamed state: the only
// part of the linearisation point that J_C^T depends on (m^eq and m^F are
// functions of rho and j, and d m^eq / d rho is constant).
template <typename T>
__device__ __forceinline__ void shifted_j(const T h[Q], const Collide<T> &p, T &jx, T &jy, T &jz) {
    jx = h[1] - h[2] + h[7] - h[8] + h[9] - h[10] + h[11] - h[12] + h[13] - h[14] + T(0.5) * p.Fx;
    jy = h[3] - h[4] + h[7] - h[8] - h[9] + h[10] + h[15] - h[16] + h[17] - h[18] + T(0.5) * p.Fy;
    jz = h[5] - h[6] + h[11] - h[12] - h[13] + h[14] + h[15] - h[16] - h[17] + h[18] + T(0.5) * p.Fz;
}

// b = D^-1 M phi (phi the streamed-back adjoint at the node).
template <typename T>
__device__ __forceinline__ void adj_moments(const T phi[Q], T b[Q]) {
    T a[Q];
    moments_of<T>(phi, a);
#pragma unroll
    for (int k = 0; k < Q; ++k) b[k] = a[k] * inv_norm<T>(k);
}

// J3 = the shifted momentum of H, component-major [3][units] (0 off fluid).
template <typename T>
__global__ void __launch_bounds__(256) k_adj_j3(const T *__restrict__ H, AdjView v, Collide<T> p,
                                                T *__restrict__ J3) {
    const uint32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= v.units) return;
    AdjUnit un;
    un.init(u, v);
    T jx = T(0), jy = T(0), jz = T(0);
    if (un.fluid) {
        T h[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) h[i] = H[(size_t)i * v.units + u];
        shifted_j<T>(h, p, jx, jy, jz);
    }
    J3[u] = jx;
    J3[(size_t)v.units + u] = jy;
    J3[2 * (size_t)v.units + u] = jz;
}

// H = streamed state (average = 0) or H = (H + streamed state) / 2 (average = 1).
// SP: sparse layout.  Its even-parity states keep every streamed value in
// the node's own slots, so those captures need no index data; odd parity
// uses the interior upstream formulas with the x faces redone, as the
// adjoint step does.
template <typename S, bool SP, bool LEAN = false>
__global__ void __launch_bounds__(256) k_adj_capture(const S *A, AdjView v, AdjState st,
                                                     float ld_scale, typename Store<S>::C *H,
                                                     int average) {
    using C = typename Store<S>::C;
    const uint32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= v.units) return;
    // all 19 loads before any store: H and A may alias as far as the
    // compiler knows, so interleaved they made 19 dependent round trips
    C val[Q];
    if (SP) {
        if (st.parity == 0) {
#pragma unroll
            for (int i = 0; i < Q; ++i) val[i] = (C)Store<S>::ld(A + (size_t)i * v.units + u, ld_scale);
        } else if (LEAN) {
            // the streamed value of direction i is where the forward odd step
            // of u reads it
            uint32_t loc[Q];
            odd_lean_locations(v.om, u, __ldg(v.om.rec + u), loc);
#pragma unroll
            for (int i = 0; i < Q; ++i)
                val[i] = v.ok(loc[i]) ? (C)Store<S>::ld(A + loc[i], ld_scale) : C(0);
        } else {
            SparseNode sn;
            sn.init(u, v.sm);
            val[0] = (C)Store<S>::ld(A + u, ld_scale);
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                uint32_t up = sn.up_interior(i);
                if (cx(i) != 0) up = min(up, v.units - 1u);  // in bounds; x faces redone below
                const size_t at = (sn.bits & (1u << i)) ? (size_t)i * v.units + u
                                                        : (size_t)opp(i) * v.units + up;
                val[i] = v.ok(at) ? (C)Store<S>::ld(A + at, ld_scale) : C(0);
            }
            if (sn.xlo || sn.xhi) {
#pragma unroll
                for (int i = 1; i < Q; ++i)
                    if (cx(i) != 0 && !(sn.bits & (1u << i))) {
                        const size_t at = (size_t)opp(i) * v.units + sn.up(i, v.sm);
                        val[i] = v.ok(at) ? (C)Store<S>::ld(A + at, ld_scale) : C(0);
                    }
            }
        }
    } else {
        AdjUnit un;
        un.init(u, v);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const size_t at = un.fluid ? streamed_loc(st, v, u, i, un) : 0;
            val[i] = un.fluid && v.ok(at) ? (C)Store<S>::ld(A + at, ld_scale) : C(0);
        }
    }
    if (average) {
        C old[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) old[i] = H[(size_t)i * v.units + u];
#pragma unroll
        for (int i = 0; i < Q; ++i) val[i] = C(0.5) * (old[i] + val[i]);
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) H[(size_t)i * v.units + u] = val[i];
}

// psi_out = J_C(h)^T S^T psi_in + coef c_{., d}.  psi_out holds the iterate
// before psi_in on entry; with `partials`, also the block sums of
// |new - that iterate|^2 (a change over two iterations, blind to a period-2
// component) and |new|^2.
// The linearisation point comes as the full streamed state H (FROM_H) or as
// its shifted momentum J3 alone (fewer bytes per iteration).
// SP: sparse layout (else dense AA/AB link words), a compile-time choice so
// that each kernel carries only its own index arithmetic.  Sparse nodes use
// the interior upstream formulas and redo the x-moving directions with the
// periodic wrap only on the x faces (as the forward odd step does).
// One unit per thread, four blocks per SM (FP32: 64 registers).  The plain
// launches of the lean index path take LBM_ADJ_LEAN_NPT units per thread,
// 256 apart, and load the next unit's record while the current one gathers
// (64 registers, four blocks per SM).  At 256^3: one unit per thread at five
// blocks per SM (48 registers, an 8-byte spill) 32.4-32.6k fluid MLUPS over
// whole adjoint runs; two units per thread 33.0k; four (56 B of spills)
// 28.9k; one unit at four or six blocks per SM 31.6k and 30.1k.
// CHK: a checking launch (residual partials, one per block of 256 units);
// its own instantiation, so that the plain launches carry none of its
// registers, and always one unit per thread.  On the lean path it runs at
// three blocks per SM (80 registers) rather than two (114): whole runs
// 33.1k -> 33.2k fluid MLUPS at 256^3.
#ifndef LBM_ADJ_LEAN_MIN_BLOCKS
#define LBM_ADJ_LEAN_MIN_BLOCKS 4
#endif
#ifndef LBM_ADJ_LEAN_NPT
#define LBM_ADJ_LEAN_NPT 2
#endif
template <typename T, bool FROM_H, bool SP, bool CHK, bool LEAN = false>
__global__ void __launch_bounds__(256, sizeof(T) == 8 ? 2
                                       : (LEAN ? (CHK ? 3 : LBM_ADJ_LEAN_MIN_BLOCKS) : (CHK ? 2 : 4)))
    k_adj_step(const T *__restrict__ H, const T *__restrict__ psi_in, T *__restrict__ psi_out,
               AdjView v, Collide<T> p, T coef, int d, double *partials) {
    constexpr int NT = (SP && LEAN && !CHK) ? LBM_ADJ_LEAN_NPT : 1;
    const uint32_t u0 = blockIdx.x * 256u * NT + threadIdx.x;
    T r[2] = {T(0), T(0)};  // residual terms of this node, in the iteration's precision
    uint2 nrec = make_uint2(0u, 0u);  // lean path: the record of the next unit
    if (SP && LEAN && u0 < v.units) nrec = __ldg(v.om.rec + u0);
#pragma unroll 1
    for (int t = 0; t < NT; ++t) {
    const uint32_t u = u0 + 256u * t;
    const uint2 rec = nrec;
    if (SP && LEAN && t + 1 < NT && u + 256u < v.units) nrec = __ldg(v.om.rec + u + 256u);
    if (u < v.units) {
        T phi[Q];
        bool fluid = true;
        // population i of x went downstream to x + c_i = x - c_opp(i), or
        // bounced back into slot opp(i) of x
        if (SP && LEAN) {
            // the forward odd step's location of direction opp(i) is slot i
            // of the node at x + c_i, or slot opp(i) of x where that voxel is
            // solid: exactly where psi_i(x + c_i) (or the bounceback value)
            // sits in the two-array layout
            uint32_t loc[Q];
            odd_lean_locations(v.om, u, rec, loc);
            phi[0] = psi_in[u];
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                const uint32_t at = loc[opp(i)];
                phi[i] = v.ok(at) ? psi_in[at] : T(0);
            }
        } else if (SP) {
            SparseNode sn;
            sn.init(u, v.sm);
            phi[0] = psi_in[u];
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                const int o = opp(i);
                // on the x faces the interior index of an x-moving direction
                // is wrong and may lie outside [0, units) (-1 or units at the
                // ends of the fluid list): clamp it, so that this load stays
                // in bounds; the value is replaced just below
                uint32_t up = sn.up_interior(o);
                if (cx(o) != 0) up = min(up, v.units - 1u);
                const size_t at = (sn.bits & (1u << o)) ? (size_t)o * v.units + u
                                                        : (size_t)i * v.units + up;
                phi[i] = v.ok(at) ? psi_in[at] : T(0);
            }
            if (sn.xlo || sn.xhi) {
#pragma unroll
                for (int i = 1; i < Q; ++i) {
                    const int o = opp(i);
                    if (cx(o) != 0 && !(sn.bits & (1u << o))) {
                        const size_t at = (size_t)i * v.units + sn.up(o, v.sm);
                        phi[i] = v.ok(at) ? psi_in[at] : T(0);
                    }
                }
            }
        } else {
            const uint32_t w = v.lw[u];
            fluid = !(w & NOT_FLUID);
            if (fluid) {
                DenseNode dn;
                dn.init(u, v.d);
                phi[0] = psi_in[u];
#pragma unroll
                for (int i = 1; i < Q; ++i) {
                    const int o = opp(i);
                    const size_t at = (w & (1u << o)) ? (size_t)o * v.units + u
                                                      : (size_t)i * v.units + dn.up(o);
                    phi[i] = v.ok(at) ? psi_in[at] : T(0);
                }
            }
        }
        if (fluid) {
            T b[Q], c[Q];
            T jx, jy, jz;
            if (FROM_H) {
                T h[Q];
#pragma unroll
                for (int i = 0; i < Q; ++i) h[i] = H[(size_t)i * v.units + u];
                shifted_j<T>(h, p, jx, jy, jz);
            } else {
                jx = H[u];
                jy = H[(size_t)v.units + u];
                jz = H[2 * (size_t)v.units + u];
            }
            adj_moments<T>(phi, b);
            // a checking launch compares with the iterate psi_out holds: its
            // 19 values are loaded here, into phi (no longer needed), all at
            // once; loaded next to their stores they made 19 dependent round
            // trips per node
            if (CHK) {
#pragma unroll
                for (int i = 0; i < Q; ++i) phi[i] = psi_out[(size_t)i * v.units + u];
            }
            const T q = p.linear ? T(0) : T(1);
            T sb[Q], kb[Q];
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                const T s = rate_of<T>(k, p);
                sb[k] = s * b[k];
                kb[k] = (T(1) - T(0.5) * s) * b[k];
                c[k] = (T(1) - s) * b[k];
            }
            c[0] = b[0] - T(11) * sb[1] + T(3) * sb[2];
            c[3] = b[3] - T(2.0 / 3.0) * sb[4] + q * (dotP<T>(0, jx, jy, jz, sb) + dotP<T>(0, p.Fx, p.Fy, p.Fz, kb));
            c[5] = b[5] - T(2.0 / 3.0) * sb[6] + q * (dotP<T>(1, jx, jy, jz, sb) + dotP<T>(1, p.Fx, p.Fy, p.Fz, kb));
            c[7] = b[7] - T(2.0 / 3.0) * sb[8] + q * (dotP<T>(2, jx, jy, jz, sb) + dotP<T>(2, p.Fx, p.Fy, p.Fz, kb));
            T out[Q];
            populations_from<T>(c, out);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const int ci = d == 0 ? cx(i) : (d == 1 ? cy(i) : cz(i));
                const T val = out[i] + coef * T(ci);
                T *dst = psi_out + (size_t)i * v.units + u;
                if (CHK) {
                    const T dv = val - phi[i];
                    r[0] += dv * dv;
                    r[1] += val * val;
                }
                *dst = val;
            }
        } else {
#pragma unroll
            for (int i = 0; i < Q; ++i) psi_out[(size_t)i * v.units + u] = T(0);
        }
    }
    }
    if (CHK) block_sum2<T>(r[0], r[1], partials);
}

// A captured chunk of the steady adjoint iteration, for one assignment of
// the two iterate buffers (cur is where the chunk starts reading).
struct AdjGraph {
    cudaGraphExec_t exec = nullptr;
    void *cur = nullptr;
    int64_t dlaunches = 0;
};

// Blocks of k_adj_step for `units` units (also its number of partials).
static unsigned adj_step_grid(uint32_t units) { return (units + 255u) / 256u; }

template <typename T, bool FROM_H>
void launch_adj_step(lbm_ctx *c, const AdjView &v, const T *H, const T *psi_in, T *psi_out,
                     const Collide<T> &p, T coef, int d, double *partials) {
    const unsigned grid = adj_step_grid(v.units);
    if (grid == 0) return;
    const bool sp = v.layout == LBM_LAYOUT_SPARSE;
    if (LBM_ADJ_LEAN && sp && v.om.rec && sizeof(T) == 4) {  // the lean index path (FP32)
        if (partials)
            k_adj_step<T, FROM_H, true, true, true><<<grid, 256, 0, c->stream>>>(
                H, psi_in, psi_out, v, p, coef, d, partials);
        else
            k_adj_step<T, FROM_H, true, false, true>
                <<<(v.units + 256u * LBM_ADJ_LEAN_NPT - 1) / (256u * LBM_ADJ_LEAN_NPT), 256, 0,
                   c->stream>>>(H, psi_in, psi_out, v, p, coef, d, nullptr);
        c->launches++;
        return;
    }
    if (partials) {
        if (sp)
            k_adj_step<T, FROM_H, true, true><<<grid, 256, 0, c->stream>>>(H, psi_in, psi_out, v, p,
                                                                           coef, d, partials);
        else
            k_adj_step<T, FROM_H, false, true><<<grid, 256, 0, c->stream>>>(H, psi_in, psi_out, v,
                                                                            p, coef, d, partials);
    } else {
        if (sp)
            k_adj_step<T, FROM_H, true, false><<<grid, 256, 0, c->stream>>>(H, psi_in, psi_out, v,
                                                                            p, coef, d, nullptr);
        else
            k_adj_step<T, FROM_H, false, false><<<grid, 256, 0, c->stream>>>(H, psi_in, psi_out, v,
                                                                             p, coef, d, nullptr);
    }
    c->launches++;
}

// Per-node gradient contributions at the converged adjoint, with psi the
// mean of the last two iterates (psi_a + psi_b) / 2:
// [0..5] dk/ds for the rate groups (e, eps, q, nu, pi, m):
//        sum_k b_k (-(m_k - meq_k) - mF_k / 2) over the group's moments;
// [6..8] dk/dF_a through the collision:
//        b_{j_a} - (2/3) b_{q_a} + q [ (1/2) dP_a(j; s b) + dP_a(j + F/2; (1 - s/2) b) ];
// [9]    the drive component of sum_x (sum_i c_i h_i + F/2) (N times the mean
//        velocity of the linearisation point).
// ACC: add the block's sums into `partials` (the transient sweep keeps one
// accumulator per block over all its steps).
// SP: sparse layout (else dense), as in k_adj_step.
template <typename T, bool ACC, bool SP, bool LEAN = false>
__global__ void __launch_bounds__(256) k_adj_grad(const T *__restrict__ H, const T *__restrict__ psi_a,
                                                  const T *__restrict__ psi_b, AdjView v,
                                                  Collide<T> p, int d, double *partials) {
    const uint32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    // per-node terms in the iteration's precision (FP64 arithmetic is scarce
    // on this GPU and this pass runs at every step of the transient
    // adjoint); block sums as in block_sum_n
    T gsum[10] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
    // psi_a == psi_b (the transient pass): 0.5 (x + x) is x exactly
    const bool same = psi_a == psi_b;
    auto psi_at = [&](size_t at) -> T {
        if (!v.ok(at)) return T(0);
        return same ? psi_a[at] : T(0.5) * (psi_a[at] + psi_b[at]);
    };
    if (u < v.units) {
        bool fluid = true;
        T phi[Q];
        // the value streamed back to u from direction i, as k_adj_step reads it
        if (SP && LEAN) {
            uint32_t loc[Q];
            odd_lean_locations(v.om, u, __ldg(v.om.rec + u), loc);
            phi[0] = psi_at(u);
#pragma unroll
            for (int i = 1; i < Q; ++i) phi[i] = psi_at(loc[opp(i)]);
        } else if (SP) {
            SparseNode sn;
            sn.init(u, v.sm);
            phi[0] = psi_at(u);
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                const int o = opp(i);
                uint32_t up = sn.up_interior(o);
                if (cx(o) != 0) up = min(up, v.units - 1u);  // in bounds; x faces redone below
                phi[i] = psi_at((sn.bits & (1u << o)) ? (size_t)o * v.units + u
                                                     : (size_t)i * v.units + up);
            }
            if (sn.xlo || sn.xhi) {
#pragma unroll
                for (int i = 1; i < Q; ++i) {
                    const int o = opp(i);
                    if (cx(o) != 0 && !(sn.bits & (1u << o)))
                        phi[i] = psi_at((size_t)i * v.units + sn.up(o, v.sm));
                }
            }
        } else {
            const uint32_t w = v.lw[u];
            fluid = !(w & NOT_FLUID);
            if (fluid) {
                DenseNode dn;
                dn.init(u, v.d);
                phi[0] = psi_at(u);
#pragma unroll
                for (int i = 1; i < Q; ++i) {
                    const int o = opp(i);
                    phi[i] = psi_at((w & (1u << o)) ? (size_t)o * v.units + u
                                                    : (size_t)i * v.units + dn.up(o));
                }
            }
        }
        if (fluid) {
            T h[Q], b[Q], m[Q], meq[Q], mF[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) h[i] = H[(size_t)i * v.units + u];
            T jx, jy, jz;
            shifted_j<T>(h, p, jx, jy, jz);
            adj_moments<T>(phi, b);
            moments_of<T>(h, m);
            eq_and_force<T>(m[0], jx, jy, jz, p, meq, mF);
            T rk[Q];
#pragma unroll
            for (int k = 0; k < Q; ++k) rk[k] = b[k] * (-(m[k] - meq[k]) - T(0.5) * mF[k]);
            gsum[0] = rk[1];
            gsum[1] = rk[2];
            gsum[2] = rk[4] + rk[6] + rk[8];
            gsum[3] = rk[9] + rk[11] + rk[13] + rk[14] + rk[15];
            gsum[4] = rk[10] + rk[12];
            gsum[5] = rk[16] + rk[17] + rk[18];
            const T q = p.linear ? T(0) : T(1);
            T sb[Q], kb[Q];
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                const T s = rate_of<T>(k, p);
                sb[k] = s * b[k];
                kb[k] = (T(1) - T(0.5) * s) * b[k];
            }
            const T ux = jx + T(0.5) * p.Fx, uy = jy + T(0.5) * p.Fy, uz = jz + T(0.5) * p.Fz;
            gsum[6] = b[3] - T(2.0 / 3.0) * b[4] +
                      q * (T(0.5) * dotP<T>(0, jx, jy, jz, sb) + dotP<T>(0, ux, uy, uz, kb));
            gsum[7] = b[5] - T(2.0 / 3.0) * b[6] +
                      q * (T(0.5) * dotP<T>(1, jx, jy, jz, sb) + dotP<T>(1, ux, uy, uz, kb));
            gsum[8] = b[7] - T(2.0 / 3.0) * b[8] +
                      q * (T(0.5) * dotP<T>(2, jx, jy, jz, sb) + dotP<T>(2, ux, uy, uz, kb));
            gsum[9] = d == 0 ? jx : (d == 1 ? jy : jz);
        }
    }
    block_sum_n<T, 10, ACC>(gsum, partials);
}

template <typename T, bool ACC>
void launch_adj_grad(lbm_ctx *c, const AdjView &v, unsigned grid, const T *H, const T *psi_a,
                     const T *psi_b, const Collide<T> &p, int d, double *partials) {
    if (LBM_ADJ_LEAN && v.layout == LBM_LAYOUT_SPARSE && v.om.rec && sizeof(T) == 4)
        k_adj_grad<T, ACC, true, true><<<grid, 256, 0, c->stream>>>(H, psi_a, psi_b, v, p, d, partials);
    else if (v.layout == LBM_LAYOUT_SPARSE)
        k_adj_grad<T, ACC, true><<<grid, 256, 0, c->stream>>>(H, psi_a, psi_b, v, p, d, partials);
    else
        k_adj_grad<T, ACC, false><<<grid, 256, 0, c->stream>>>(H, psi_a, psi_b, v, p, d, partials);
}

// Fixed-order sum of NV-component partials by one block.
template <int NV>
__global__ void __launch_bounds__(1024) k_sum_partials(const double *__restrict__ partials, int nblk,
                                                        double *out) {
    __shared__ double sm[NV][1024];
    double acc[NV];
#pragma unroll
    for (int a = 0; a < NV; ++a) acc[a] = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x)
#pragma unroll
        for (int a = 0; a < NV; ++a) acc[a] += partials[(size_t)NV * b + a];
#pragma unroll
    for (int a = 0; a < NV; ++a) sm[a][threadIdx.x] = acc[a];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
#pragma unroll
            for (int a = 0; a < NV; ++a) sm[a][threadIdx.x] += sm[a][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < NV) out[threadIdx.x] = sm[threadIdx.x][0];
}

SparseMap sparse_map(const lbm_ctx *c);
OddMap odd_map(const lbm_ctx *c);

static AdjView make_adj_view(const lbm_ctx *c) {
    AdjView v;
    v.layout = c->opt.layout;
    v.units = (uint32_t)(c->opt.layout == LBM_LAYOUT_SPARSE ? c->Nf : c->N);
    v.lw = c->d_lw;
    v.sm = sparse_map(c);
    v.d = Dims{c->Lx, c->Ly, c->Lz, (uint32_t)c->N};
    v.om = odd_map(c);  // rec is null unless the sparse layout built the lean tables
    return v;
}

template <typename T>
static Collide<T> collide_params(const lbm_ctx *c) {
    return make_collide<T>(c->s, c->F, c->opt.linear_eq, c->opt.collision == 0);
}

int launch_step(lbm_ctx *c, bool reduce);

template <typename T>
static void capture(lbm_ctx *c, const AdjView &v, unsigned grid, T *H, int average) {
    const AdjState st{c->opt.layout, (int)(c->steps & 1)};
    const float lds = c->fp16_scale > 0.f ? 1.0f / c->fp16_scale : 1.0f;
    const void *A = c->opt.layout == LBM_LAYOUT_AB ? c->d_pop[c->cur] : c->d_pop[0];
    const bool sp = c->opt.layout == LBM_LAYOUT_SPARSE;
    switch (c->opt.precision) {
    case LBM_FP64:
        if (sp)
            k_adj_capture<double, true><<<grid, 256, 0, c->stream>>>((const double *)A, v, st, lds,
                                                                     (double *)H, average);
        else
            k_adj_capture<double, false><<<grid, 256, 0, c->stream>>>((const double *)A, v, st, lds,
                                                                      (double *)H, average);
        break;
    case LBM_FP32_SHIFTED:
        if (sp && v.om.rec && LBM_ADJ_LEAN)
            k_adj_capture<float, true, true><<<grid, 256, 0, c->stream>>>((const float *)A, v, st,
                                                                          lds, (float *)H, average);
        else if (sp)
            k_adj_capture<float, true><<<grid, 256, 0, c->stream>>>((const float *)A, v, st, lds,
                                                                    (float *)H, average);
        else
            k_adj_capture<float, false><<<grid, 256, 0, c->stream>>>((const float *)A, v, st, lds,
                                                                     (float *)H, average);
        break;
    default:
        if (sp && v.om.rec && LBM_ADJ_LEAN)
            k_adj_capture<__half, true, true><<<grid, 256, 0, c->stream>>>(
                (const __half *)A, v, st, lds, (float *)H, average);
        else if (sp)
            k_adj_capture<__half, true><<<grid, 256, 0, c->stream>>>((const __half *)A, v, st, lds,
                                                                     (float *)H, average);
        else
            k_adj_capture<__half, false><<<grid, 256, 0, c->stream>>>((const __half *)A, v, st, lds,
                                                                      (float *)H, average);
        break;
    }
    c->launches++;
}

// Runs the adjoint iteration and the gradient pass in arithmetic type T.
// sums[0..9] receive the raw gradient sums (see k_adj_grad); *iters and
// *resid the iteration count and final relative residual.  The context
// advances one step (the linearisation point is a two-step mean).
template <typename T>
static int adjoint_run(lbm_ctx *c, double tol, int64_t max_iter, int d, double coef,
                       double sums[10], int64_t *iters, double *resid) {
    const AdjView v = make_adj_view(c);
    const size_t bytes = sizeof(T) * Q * (size_t)v.units;
    T *H = nullptr, *cur = nullptr, *prev = nullptr, *J3 = nullptr;
    double *part = nullptr, *dsum = nullptr;
    const unsigned grid = (unsigned)((v.units + 255) / 256);
    cudaError_t e = cudaMalloc(&H, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&J3, sizeof(T) * 3 * (size_t)(v.units > 0 ? v.units : 1));
    if (e == cudaSuccess) e = cudaMalloc(&cur, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&prev, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&part, sizeof(double) * 10 * (size_t)(grid > 0 ? grid : 1));
    if (e == cudaSuccess) e = cudaMalloc(&dsum, sizeof(double) * 10);
    auto cleanup = [&]() {
        cudaFree(H);
        cudaFree(J3);
        cudaFree(cur);
        cudaFree(prev);
        cudaFree(part);
        cudaFree(dsum);
    };
    if (e != cudaSuccess) {
        cleanup();
        return launch_error(e);
    }
    const Collide<T> p = collide_params<T>(c);
    *iters = 0;
    *resid = NAN;
    for (int a = 0; a < 10; ++a) sums[a] = 0.0;
    if (grid > 0) {
        // H = (streamed state now + streamed state after one more step) / 2
        capture<T>(c, v, grid, H, 0);
        launch_step(c, false);
        capture<T>(c, v, grid, H, 1);
        // the iteration needs the linearisation point only through its momentum
        k_adj_j3<T><<<grid, 256, 0, c->stream>>>(H, v, p, J3);
        c->launches++;
        // psi_{-1} = psi_0 = 0: the first step gives psi_1 = dJ/dh
        e = cudaMemsetAsync(cur, 0, bytes, c->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(prev, 0, bytes, c->stream);
        const int64_t K = c->opt.check_interval > 0 ? c->opt.check_interval : 100;
        const int nstep_part = (int)adj_step_grid(v.units);
        double host[2];
        // A whole chunk of K iterations (the last one checking the residual)
        // is captured once per pair of iterate buffers as a CUDA graph and
        // replayed; K even needs one graph, K odd two.
        AdjGraph graphs[2];
        bool unstable = false;
        NvtxRange range("lbm_adjoint iterations");
        while (e == cudaSuccess && *iters < max_iter) {
            if (K >= 2 && *iters % K == 0 && max_iter - *iters >= K) {
                AdjGraph *G = nullptr;
                for (AdjGraph &g : graphs)
                    if (g.exec && g.cur == (void *)cur) G = &g;
                if (!G) {
                    AdjGraph &slot = graphs[graphs[0].exec ? 1 : 0];
                    if (slot.exec) cudaGraphExecDestroy(slot.exec);
                    slot = AdjGraph{};
                    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
                    if (cudaStreamIsCapturing(c->stream, &cs) == cudaSuccess &&
                        cs == cudaStreamCaptureStatusNone &&
                        cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) ==
                            cudaSuccess) {
                        const int64_t l0 = c->launches;
                        T *a = cur, *b = prev;
                        for (int64_t t = 0; t < K; ++t) {
                            launch_adj_step<T, false>(c, v, J3, a, b, p, (T)coef, d,
                                                      t + 1 == K ? part : nullptr);
                            T *x = a;
                            a = b;
                            b = x;
                        }
                        k_sum_partials<2><<<1, 1024, 0, c->stream>>>(part, nstep_part, dsum);
                        c->launches++;
                        slot.dlaunches = c->launches - l0;
                        c->launches = l0;
                        cudaGraph_t graph = nullptr;
                        cudaError_t ce = cudaStreamEndCapture(c->stream, &graph);
                        if (ce == cudaSuccess) ce = cudaGraphInstantiate(&slot.exec, graph, 0);
                        if (graph) cudaGraphDestroy(graph);
                        if (ce != cudaSuccess) {
                            cudaGetLastError();
                            slot.exec = nullptr;
                        } else {
                            slot.cur = cur;
                            G = &slot;
                        }
                    } else {
                        cudaGetLastError();
                    }
                }
                if (G) {
                    e = cudaGraphLaunch(G->exec, c->stream);
                    if (e != cudaSuccess) break;
                    c->launches += G->dlaunches;
                    if (K % 2) {
                        T *x = cur;
                        cur = prev;
                        prev = x;
                    }
                    *iters += K;
                    e = cudaMemcpyAsync(host, dsum, sizeof host, cudaMemcpyDeviceToHost, c->stream);
                    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
                    if (e != cudaSuccess) break;
                    *resid = host[1] > 0.0 ? sqrt(host[0] / host[1]) : 0.0;
                    if (!isfinite(*resid)) {
                        unstable = true;
                        break;
                    }
                    if (*resid <= tol) break;
                    continue;
                }
            }
            const bool check = *iters >= 1 && (((*iters + 1) % K == 0) || (*iters + 1 == max_iter));
            // prev <- J^T S^T cur + g (prev held the iterate before cur)
            launch_adj_step<T, false>(c, v, J3, cur, prev, p, (T)coef, d, check ? part : nullptr);
            T *t = cur;
            cur = prev;
            prev = t;
            ++*iters;
            if (check) {
                k_sum_partials<2><<<1, 1024, 0, c->stream>>>(part, nstep_part, dsum);
                c->launches++;
                e = cudaMemcpyAsync(host, dsum, sizeof host, cudaMemcpyDeviceToHost, c->stream);
                if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
                if (e != cudaSuccess) break;
                *resid = host[1] > 0.0 ? sqrt(host[0] / host[1]) : 0.0;
                if (!isfinite(*resid)) {
                    unstable = true;
                    break;
                }
                if (*resid <= tol) break;
            }
        }
        for (AdjGraph &g : graphs)
            if (g.exec) cudaGraphExecDestroy(g.exec);
        if (unstable) {
            cleanup();
            return LBM_EUNSTABLE;
        }
        if (e == cudaSuccess) {
            launch_adj_grad<T, false>(c, v, grid, H, cur, prev, p, d, part);
            k_sum_partials<10><<<1, 1024, 0, c->stream>>>(part, (int)grid, dsum);
            c->launches += 2;
            e = cudaMemcpyAsync(sums, dsum, sizeof(double) * 10, cudaMemcpyDeviceToHost, c->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        }
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    cleanup();
    return launch_error(e);
}

// Transient adjoint: the gradient of k after n more steps, J = k(h_{n+1}),
// by reverse accumulation.  h_t is the state step t collides; with
// phi_{n+1} = dJ/dh and phi_t = J_C(h_t)^T S^T phi_{t+1}, the gradient sums
// are those of k_adj_grad at (h_t, phi_{t+1}) added over t.  The forward
// states are not all kept: the raw population array is saved every
// C = ceil(sqrt(n)) steps; the reverse sweep restores each checkpoint, steps
// through its segment again capturing h_t, and walks the segment backwards.
// About 2 sqrt(n) fields of device memory.  sums[9] receives N U_d of
// h_{n+1}; the context ends n steps on, at the forward sweep's final state.
template <typename T>
static int transient_run(lbm_ctx *c, int64_t n, int d, double coef, double sums[10]) {
    NvtxRange range("lbm_adjoint_transient");
    const AdjView v = make_adj_view(c);
    const unsigned grid = (unsigned)((v.units + 255) / 256);
    for (int a = 0; a < 10; ++a) sums[a] = 0.0;
    if (grid == 0) {
        for (int64_t t = 0; t < n; ++t) launch_step(c, false);
        return launch_error(cudaGetLastError());
    }
    const int64_t C = (int64_t)ceil(sqrt((double)n));
    const int64_t nseg = (n + C - 1) / C;
    const size_t fieldT = (size_t)Q * v.units;            // elements of one adjoint field
    const size_t sbytes = c->elem * (size_t)Q * v.units;  // bytes of one population state
    T *Hbuf = nullptr, *psi = nullptr, *nxt = nullptr;
    unsigned char *ckpt = nullptr;
    double *part = nullptr, *acc = nullptr, *dsum = nullptr;
    cudaError_t e = cudaMalloc(&Hbuf, sizeof(T) * fieldT * (size_t)C);
    if (e == cudaSuccess) e = cudaMalloc(&ckpt, sbytes * (size_t)(nseg + 1));
    if (e == cudaSuccess) e = cudaMalloc(&psi, sizeof(T) * fieldT);
    if (e == cudaSuccess) e = cudaMalloc(&nxt, sizeof(T) * fieldT);
    if (e == cudaSuccess) e = cudaMalloc(&part, sizeof(double) * 10 * (size_t)grid);
    if (e == cudaSuccess) e = cudaMalloc(&acc, sizeof(double) * 10 * (size_t)grid);
    if (e == cudaSuccess) e = cudaMalloc(&dsum, sizeof(double) * 20);
    auto cleanup = [&]() {
        cudaFree(Hbuf);
        cudaFree(ckpt);
        cudaFree(psi);
        cudaFree(nxt);
        cudaFree(part);
        cudaFree(acc);
        cudaFree(dsum);
    };
    if (e != cudaSuccess) {
        cleanup();
        cudaGetLastError();  // clear the failed allocation
        return LBM_ENOMEM;
    }
    std::vector<int64_t> ck_steps(nseg + 1);
    std::vector<int> ck_cur(nseg + 1);
    auto state = [&]() -> void * {
        return c->opt.layout == LBM_LAYOUT_AB ? c->d_pop[c->cur] : c->d_pop[0];
    };
    auto save = [&](int64_t k) {
        ck_steps[k] = c->steps;
        ck_cur[k] = c->cur;
        return cudaMemcpyAsync(ckpt + sbytes * (size_t)k, state(), sbytes, cudaMemcpyDeviceToDevice,
                               c->stream);
    };
    auto restore = [&](int64_t k) {
        c->steps = ck_steps[k];
        c->cur = ck_cur[k];
        return cudaMemcpyAsync(state(), ckpt + sbytes * (size_t)k, sbytes, cudaMemcpyDeviceToDevice,
                               c->stream);
    };
    const Collide<T> p = collide_params<T>(c);
    // forward sweep with checkpoints
    for (int64_t sg = 0; sg < nseg && e == cudaSuccess; ++sg) {
        e = save(sg);
        const int64_t len = (sg + 1) * C <= n ? C : n - sg * C;
        for (int64_t t = 0; t < len; ++t) launch_step(c, false);
    }
    if (e == cudaSuccess) e = save(nseg);
    // seed phi_{n+1} = coef c_d at fluid nodes (one adjoint step of a zero
    // field, with the captured final state as a finite linearisation point),
    // and N U_d of h_{n+1}
    if (e == cudaSuccess) {
        capture<T>(c, v, grid, Hbuf, 0);
        e = cudaMemsetAsync(nxt, 0, sizeof(T) * fieldT, c->stream);
    }
    if (e == cudaSuccess) {
        launch_adj_step<T, true>(c, v, Hbuf, nxt, psi, p, (T)coef, d, nullptr);
        launch_adj_grad<T, false>(c, v, grid, Hbuf, nxt, nxt, p, d, part);
        k_sum_partials<10><<<1, 1024, 0, c->stream>>>(part, (int)grid, dsum + 10);
        c->launches += 2;
        // the steps t < n add their block sums into acc, summed once at the end
        e = cudaMemsetAsync(acc, 0, sizeof(double) * 10 * (size_t)grid, c->stream);
    }
    // reverse sweep, segment by segment
    for (int64_t sg = nseg - 1; sg >= 0 && e == cudaSuccess; --sg) {
        e = restore(sg);
        const int64_t len = (sg + 1) * C <= n ? C : n - sg * C;
        for (int64_t t = 0; t < len; ++t) {
            capture<T>(c, v, grid, Hbuf + fieldT * (size_t)t, 0);
            launch_step(c, false);
        }
        for (int64_t t = len - 1; t >= 0; --t) {
            const T *H = Hbuf + fieldT * (size_t)t;
            launch_adj_grad<T, true>(c, v, grid, H, psi, psi, p, d, acc);
            launch_adj_step<T, true>(c, v, H, psi, nxt, p, (T)0, d, nullptr);
            c->launches += 1;
            T *tmp = psi;
            psi = nxt;
            nxt = tmp;
        }
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = restore(nseg);
    if (e == cudaSuccess) {
        k_sum_partials<10><<<1, 1024, 0, c->stream>>>(acc, (int)grid, dsum);
        c->launches++;
    }
    double host[20];
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(host, dsum, sizeof host, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) {
        // steps t < n: components 0..8 summed over blocks and steps; step n
        // contributes only N U_d of the final state (component 9)
        for (int a = 0; a < 9; ++a) sums[a] = host[a];
        sums[9] = host[10 + 9];
    }
    cleanup();
    return launch_error(e);
}

int transient_sums(lbm_ctx *c, int64_t n, int d, double coef, double sums[10]) {
    if (c->opt.precision == LBM_FP64) return transient_run<double>(c, n, d, coef, sums);
    return transient_run<float>(c, n, d, coef, sums);
}

int adjoint_sums(lbm_ctx *c, double tol, int64_t max_iter, int d, double coef, double sums[10],
                 int64_t *iters, double *resid) {
    if (c->opt.precision == LBM_FP64)
        return adjoint_run<double>(c, tol, max_iter, d, coef, sums, iters, resid);
    return adjoint_run<float>(c, tol, max_iter, d, coef, sums, iters, resid);
}

}  // namespace lbm
