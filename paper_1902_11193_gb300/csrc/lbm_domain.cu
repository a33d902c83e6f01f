// Bounded domains (Sec. 2.4) for the AB layout: x faces with prescribed
// density (Zou-He) and y and/or z faces as symmetry (mirror) planes.
//
// Real samples are not periodic: the paper pads the inlet and outlet with
// fluid layers, mirrors the lateral faces and drives the flow by a density
// difference.  This file holds the stream-collide and the streamed-state
// velocity for such a domain; the periodic kernels are untouched.  The pull
// at fluid node x for direction j:
// - source x - c_j outside a mirror face: the specular image of the
//   population that left the neighbouring node along the mirrored
//   direction, i.e. the source keeps the node's y (or z) and direction j's
//   y (or z) component is reversed;
// - source outside an x face with prescribed density: unknown after the
//   pull; set by non-equilibrium bounceback,
//   g_j = g_opp(j) + 6 w_j c_jx j_x - c_jy N_y - c_jz N_z,
//   with j_x = n_x (drho - S_0 - 2 S_out) from the prescribed density
//   deviation drho, the in-plane populations S_0 and those leaving through
//   the face S_out (inward normal n_x), and N_t half the tangential momentum
//   of the in-plane populations, so that the node carries the prescribed
//   density and no tangential momentum (the shifted populations g = f - w
//   keep these formulas: the rest weights add 2/3 in the plane and 1/6 on
//   each side);
// - otherwise halfway bounceback where the (mirrored) source voxel is solid.
#include "lbm_step.cuh"

namespace lbm {

__host__ __device__ constexpr int dir_of(int x, int y, int z) {
    int d = -1;
    for (int j = 0; j < Q; ++j)
        if (cx(j) == x && cy(j) == y && cz(j) == z) d = j;
    return d;
}
__host__ __device__ constexpr int mirror_y(int j) { return dir_of(cx(j), -cy(j), cz(j)); }
__host__ __device__ constexpr int mirror_z(int j) { return dir_of(cx(j), cy(j), -cz(j)); }

struct Domain {
    int pressure_x;            // Zou-He faces at x = 0 (inlet) and x = Lx - 1 (outlet)
    int symmetry;              // bit 0: y faces, bit 1: z faces are mirror planes
    double drho_in, drho_out;  // prescribed densities minus rho0
};

template <typename S>
__device__ __forceinline__ void bounded_pull(const S *__restrict__ A, const uint8_t *__restrict__ mask,
                                             const Dims &d, const Domain &dom, int x, int y, int z,
                                             uint32_t n, float lds, typename Store<S>::C g[Q],
                                             int *flag) {
    using C = typename Store<S>::C;
    uint32_t unknown = 0;
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        int xs = x - cx(j), ys = y - cy(j), zs = z - cz(j);
        if (dom.pressure_x && (xs < 0 || xs >= d.Lx)) {
            unknown |= 1u << j;
            g[j] = C(0);
            continue;
        }
        xs = xs < 0 ? xs + d.Lx : (xs >= d.Lx ? xs - d.Lx : xs);
        bool my = false, mz = false;
        if ((dom.symmetry & 1) && (ys < 0 || ys >= d.Ly)) {
            ys = y;
            my = true;
        } else {
            ys = ys < 0 ? ys + d.Ly : (ys >= d.Ly ? ys - d.Ly : ys);
        }
        if ((dom.symmetry & 2) && (zs < 0 || zs >= d.Lz)) {
            zs = z;
            mz = true;
        } else {
            zs = zs < 0 ? zs + d.Lz : (zs >= d.Lz ? zs - d.Lz : zs);
        }
        const int dir = my ? (mz ? mirror_z(mirror_y(j)) : mirror_y(j)) : (mz ? mirror_z(j) : j);
        const uint32_t s = (uint32_t)xs + (uint32_t)d.Lx * ((uint32_t)ys + (uint32_t)d.Ly * (uint32_t)zs);
        const bool solid = in_range(s, d.N, flag) ? mask[s] != 0 : true;
        const size_t at = solid ? (size_t)opp(j) * d.N + n : (size_t)dir * d.N + s;
        g[j] = in_range(at, (uint64_t)Q * d.N, flag) ? Store<S>::ld(A + at, lds) : C(0);
    }
    if (unknown) {
        const int nx = x == 0 ? 1 : -1;
        const C drho = (C)(x == 0 ? dom.drho_in : dom.drho_out);
        C s0 = C(0), sout = C(0), Ny = C(0), Nz = C(0);
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            if (cx(j) == 0) {
                s0 += g[j];
                Ny += C(0.5 * cy(j)) * g[j];
                Nz += C(0.5 * cz(j)) * g[j];
            } else if (cx(j) == -nx) {
                sout += g[j];
            }
        }
        const C jx = C(nx) * (drho - s0 - C(2) * sout);
#pragma unroll
        for (int j = 0; j < Q; ++j)
            if (unknown & (1u << j))
                g[j] = g[opp(j)] + C(6.0 * weight(j) * cx(j)) * jx - C(cy(j)) * Ny - C(cz(j)) * Nz;
    }
}

// Per-block FP64 partial sums of the shifted velocity, fixed order.
__device__ __forceinline__ void block_sum3(double v[3], double *partials) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[a] += __shfl_down_sync(0xffffffffu, v[a], o);
    __shared__ double sm[32][3];
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int a = 0; a < 3; ++a) sm[threadIdx.x >> 5][a] = v[a];
    __syncthreads();
    if (threadIdx.x < 3) {
        double acc = 0.0;
        for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) acc += sm[w][threadIdx.x];
        partials[3 * (size_t)blockIdx.x + threadIdx.x] = acc;
    }
}

__device__ __forceinline__ void node_xyz(uint32_t n, const Dims &d, int &x, int &y, int &z) {
    const uint32_t t = n / (uint32_t)d.Lx;
    x = (int)(n - t * (uint32_t)d.Lx);
    z = (int)(t / (uint32_t)d.Ly);
    y = (int)(t - (uint32_t)z * (uint32_t)d.Ly);
}

template <typename S, int K>
__global__ void __launch_bounds__(256) k_ab_bounded(const S *__restrict__ src, S *__restrict__ dst,
                                                    const uint8_t *__restrict__ mask, Dims d,
                                                    Domain dom, Collide<typename Store<S>::C> p,
                                                    float lds, float sts, double *partials, int *flag) {
    using C = typename Store<S>::C;
    const uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
    const bool fluid = n < d.N && !mask[n];
    C jx = C(0), jy = C(0), jz = C(0);
    if (fluid) {
        int x, y, z;
        node_xyz(n, d, x, y, z);
        C g[Q];
        bounded_pull<S>(src, mask, d, dom, x, y, z, n, lds, g, flag);
        collide_as<K, C>(g, p, jx, jy, jz);
#pragma unroll
        for (int i = 0; i < Q; ++i) Store<S>::st(dst + (size_t)i * d.N + n, g[i], sts);
    }
    if (partials) {
        double v[3] = {fluid ? (double)jx : 0.0, fluid ? (double)jy : 0.0, fluid ? (double)jz : 0.0};
        if (fluid && !isfinite(v[0] + v[1] + v[2])) atomicOr(flag, 1);
        block_sum3(v, partials);
    }
}

// Streamed-state velocity u = sum c g + F/2 (0 in solids): field and/or
// per-block partial sums.
template <typename S>
__global__ void __launch_bounds__(256) k_velocity_bounded(const S *__restrict__ A,
                                                          const uint8_t *__restrict__ mask, Dims d,
                                                          Domain dom, double Fx, double Fy, double Fz,
                                                          float lds, double *u_out, double *partials,
                                                          int *flag) {
    using C = typename Store<S>::C;
    const uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
    const bool fluid = n < d.N && !mask[n];
    double v[3] = {0.0, 0.0, 0.0};
    if (fluid) {
        int x, y, z;
        node_xyz(n, d, x, y, z);
        C g[Q];
        bounded_pull<S>(A, mask, d, dom, x, y, z, n, lds, g, flag);
#pragma unroll
        for (int j = 1; j < Q; ++j) {
            v[0] += cx(j) * (double)g[j];
            v[1] += cy(j) * (double)g[j];
            v[2] += cz(j) * (double)g[j];
        }
        v[0] += 0.5 * Fx;
        v[1] += 0.5 * Fy;
        v[2] += 0.5 * Fz;
        if (u_out)
#pragma unroll
            for (int a = 0; a < 3; ++a) u_out[(size_t)a * d.N + n] = v[a];
    }
    if (partials) block_sum3(v, partials);
}

static Domain domain_of(const lbm_ctx *c) {
    return Domain{c->opt.pressure_x, c->opt.symmetry, c->opt.rho_in - 1.0, c->opt.rho_out - 1.0};
}

template <typename S>
int step_bounded_t(lbm_ctx *c, bool reduce) {
    using C = typename Store<S>::C;
    const Collide<C> p = make_collide<C>(c->s, c->F, c->opt.linear_eq, c->opt.collision == 0);
    const float lds = c->fp16_scale > 0.f ? 1.0f / c->fp16_scale : 1.0f;
    const float sts = c->fp16_scale > 0.f ? c->fp16_scale : 1.0f;
    const Dims d{c->Lx, c->Ly, c->Lz, (uint32_t)c->N};
    const unsigned grid = (unsigned)((c->N + 255) / 256);
    if (p.trt)
        k_ab_bounded<S, kCollideTrt><<<grid, 256, 0, c->stream>>>(
            (const S *)c->d_pop[c->cur], (S *)c->d_pop[1 - c->cur], c->d_mask, d, domain_of(c), p,
            lds, sts, reduce ? c->d_partials : nullptr, c->d_flag);
    else
        k_ab_bounded<S, kCollideMrt><<<grid, 256, 0, c->stream>>>(
            (const S *)c->d_pop[c->cur], (S *)c->d_pop[1 - c->cur], c->d_mask, d, domain_of(c), p,
            lds, sts, reduce ? c->d_partials : nullptr, c->d_flag);
    c->cur = 1 - c->cur;
    c->launches++;
    c->steps++;
    return reduce ? (int)grid : 0;
}

template <typename S>
int velocity_bounded_t(lbm_ctx *c, double *u_dev, bool reduce) {
    const float lds = c->fp16_scale > 0.f ? 1.0f / c->fp16_scale : 1.0f;
    const Dims d{c->Lx, c->Ly, c->Lz, (uint32_t)c->N};
    const unsigned grid = (unsigned)((c->N + 255) / 256);
    k_velocity_bounded<S><<<grid, 256, 0, c->stream>>>((const S *)c->d_pop[c->cur], c->d_mask, d,
                                                       domain_of(c), c->F[0], c->F[1], c->F[2], lds,
                                                       u_dev, reduce ? c->d_partials : nullptr,
                                                       c->d_flag);
    c->launches++;
    return (int)grid;
}

int launch_step_bounded(lbm_ctx *c, bool reduce) {
    switch (c->opt.precision) {
    case LBM_FP64: return step_bounded_t<double>(c, reduce);
    case LBM_FP32_SHIFTED: return step_bounded_t<float>(c, reduce);
    default: return step_bounded_t<__half>(c, reduce);
    }
}

int launch_velocity_bounded(lbm_ctx *c, double *u_dev, bool reduce) {
    switch (c->opt.precision) {
    case LBM_FP64: return velocity_bounded_t<double>(c, u_dev, reduce);
    case LBM_FP32_SHIFTED: return velocity_bounded_t<float>(c, u_dev, reduce);
    default: return velocity_bounded_t<__half>(c, u_dev, reduce);
    }
}

}  // namespace lbm
