// The D3Q19 MRT collision with Guo forcing for one node, on shifted
// populations g_i = f_i - w_i (rho0 = 1), and the transforms it is built of.
//
// Method (Sec. 2.2.1): m = M f; rho = m0; j = (m3, m5, m7) + F/2 (shifted
// velocity); m* = m - S (m - m^eq) + (I - S/2) m^F (eq. MRT-LBE with the
// post-collision moments); f* = M^-1 m*.  M is the orthogonal d'Humieres
// basis in the paper's moment order; here both transforms are evaluated in
// factored form from opposite-pair sums and differences (about 200 flops per
// node instead of two dense 19x19 products), and M^-1 = M^T D^-1 uses the
// row norms D.  Equilibrium moments follow eq. (MRT Equi) read as the
// projection of the second-order equilibrium (m1 = -11 rho + 19 j.j,
// m9 = 2jx^2 - jy^2 - jz^2, m10 = -m9/2, m12 = -m11/2); the forcing moments
// m^F = M F_i of eq. (Guo_Forcing) are applied in closed form.
// Shifting only removes M w = (1, -11, 3, 0, ...), i.e. the rho-proportional
// parts of m0, m1, m2, so rho enters as the deviation m0(g).
//
// Moment index: 0 rho, 1 e, 2 eps, 3 jx, 4 qx, 5 jy, 6 qy, 7 jz, 8 qz,
// 9 3pxx, 10 3pixx, 11 pww, 12 piww, 13 pxy, 14 pyz, 15 pxz, 16 mx, 17 my,
// 18 mz.
#pragma once

#include "lbm_internal.cuh"

namespace lbm {

// Squared row norms D_k of M.
template <typename T>
__device__ __forceinline__ T inv_norm(int k) {
    return k == 0 ? T(1.0 / 19.0)
         : k == 1 ? T(1.0 / 2394.0)
         : k == 2 ? T(1.0 / 252.0)
         : (k == 3 || k == 5 || k == 7) ? T(0.1)
         : (k == 4 || k == 6 || k == 8) ? T(0.025)
         : k == 9 ? T(1.0 / 36.0)
         : k == 10 ? T(1.0 / 72.0)
         : k == 11 ? T(1.0 / 12.0)
         : k == 12 ? T(1.0 / 24.0)
         : k <= 15 ? T(0.25)
                   : T(0.125);
}

// m = M g.
template <typename T>
__device__ __forceinline__ void moments_of(const T g[Q], T m[Q]) {
    const T sx = g[1] + g[2], dx = g[1] - g[2];
    const T sy = g[3] + g[4], dy = g[3] - g[4];
    const T sz = g[5] + g[6], dz = g[5] - g[6];
    const T s1 = g[7] + g[8], d1 = g[7] - g[8];        // (1, 1, 0)
    const T s2 = g[9] + g[10], d2 = g[9] - g[10];      // (1,-1, 0)
    const T s3 = g[11] + g[12], d3 = g[11] - g[12];    // (1, 0, 1)
    const T s4 = g[13] + g[14], d4 = g[13] - g[14];    // (1, 0,-1)
    const T s5 = g[15] + g[16], d5 = g[15] - g[16];    // (0, 1, 1)
    const T s6 = g[17] + g[18], d6 = g[17] - g[18];    // (0, 1,-1)
    const T sa = sx + sy + sz;
    const T sxy = s1 + s2, sxz = s3 + s4, syz = s5 + s6;
    const T se = sxy + sxz + syz;
    m[0] = g[0] + sa + se;
    m[1] = T(-30) * g[0] - T(11) * sa + T(8) * se;
    m[2] = T(12) * g[0] - T(4) * sa + se;
    const T ex = d1 + d2 + d3 + d4;  // edge part of the x-odd moments
    const T ey = d1 - d2 + d5 + d6;
    const T ez = d3 - d4 + d5 - d6;
    m[3] = dx + ex;
    m[4] = T(-4) * dx + ex;
    m[5] = dy + ey;
    m[6] = T(-4) * dy + ey;
    m[7] = dz + ez;
    m[8] = T(-4) * dz + ez;
    m[9] = T(2) * sx - sy - sz + sxy + sxz - T(2) * syz;
    m[10] = T(-4) * sx + T(2) * (sy + sz) + sxy + sxz - T(2) * syz;
    m[11] = sy - sz + sxy - sxz;
    m[12] = T(2) * (sz - sy) + sxy - sxz;
    m[13] = s1 - s2;
    m[14] = s5 - s6;
    m[15] = s3 - s4;
    m[16] = d1 + d2 - d3 - d4;
    m[17] = d5 + d6 - d1 + d2;
    m[18] = d3 - d4 - d5 + d6;
}

// g = M^T a (so g = M^-1 m for a_k = m_k / D_k).
template <typename T>
__device__ __forceinline__ void populations_from(const T a[Q], T g[Q]) {
    g[0] = a[0] - T(30) * a[1] + T(12) * a[2];
    const T axis = a[0] - T(11) * a[1] - T(4) * a[2];
    const T bx = axis + T(2) * a[9] - T(4) * a[10];
    const T ox = a[3] - T(4) * a[4];
    g[1] = bx + ox;
    g[2] = bx - ox;
    const T by = axis - a[9] + T(2) * a[10] + a[11] - T(2) * a[12];
    const T oy = a[5] - T(4) * a[6];
    g[3] = by + oy;
    g[4] = by - oy;
    const T bz = axis - a[9] + T(2) * a[10] - a[11] + T(2) * a[12];
    const T oz = a[7] - T(4) * a[8];
    g[5] = bz + oz;
    g[6] = bz - oz;
    const T edge = a[0] + T(8) * a[1] + a[2];
    const T ox2 = a[3] + a[4], oy2 = a[5] + a[6], oz2 = a[7] + a[8];
    const T bxy = edge + a[9] + a[10] + a[11] + a[12];
    const T t1 = ox2 + oy2 + a[16] - a[17];
    g[7] = bxy + a[13] + t1;
    g[8] = bxy + a[13] - t1;
    const T t2 = ox2 - oy2 + a[16] + a[17];
    g[9] = bxy - a[13] + t2;
    g[10] = bxy - a[13] - t2;
    const T bxz = edge + a[9] + a[10] - a[11] - a[12];
    const T t3 = ox2 + oz2 - a[16] + a[18];
    g[11] = bxz + a[15] + t3;
    g[12] = bxz + a[15] - t3;
    const T t4 = ox2 - oz2 - a[16] - a[18];
    g[13] = bxz - a[15] + t4;
    g[14] = bxz - a[15] - t4;
    const T byz = edge - T(2) * (a[9] + a[10]);
    const T t5 = oy2 + oz2 + a[17] - a[18];
    g[15] = byz + a[14] + t5;
    g[16] = byz + a[14] - t5;
    const T t6 = oy2 - oz2 + a[17] + a[18];
    g[17] = byz - a[14] + t6;
    g[18] = byz - a[14] - t6;
}

// Relaxation rate of moment k.
template <typename T>
__device__ __forceinline__ T rate_of(int k, const Collide<T> &p) {
    return (k == 0 || k == 3 || k == 5 || k == 7) ? T(0)
         : k == 1 ? p.se
         : k == 2 ? p.seps
         : (k == 4 || k == 6 || k == 8) ? p.sq
         : (k == 10 || k == 12) ? p.spi
         : k >= 16 ? p.sm
                   : p.snu;
}

// Equilibrium moments (shifted: rho is the deviation) and forcing moments
// for shifted momentum j (u = j / rho0, rho0 = 1).
template <typename T>
__device__ __forceinline__ void eq_and_force(T rho, T jx, T jy, T jz, const Collide<T> &p,
                                             T meq[Q], T mF[Q]) {
    const T q = p.linear ? T(0) : T(1);
    const T jj = q * (jx * jx + jy * jy + jz * jz);
    const T qxx = q * (T(2) * jx * jx - jy * jy - jz * jz);
    const T qww = q * (jy * jy - jz * jz);
    meq[0] = rho;
    meq[1] = T(-11) * rho + T(19) * jj;
    meq[2] = T(3) * rho - T(5.5) * jj;
    meq[3] = jx;
    meq[4] = T(-2.0 / 3.0) * jx;
    meq[5] = jy;
    meq[6] = T(-2.0 / 3.0) * jy;
    meq[7] = jz;
    meq[8] = T(-2.0 / 3.0) * jz;
    meq[9] = qxx;
    meq[10] = T(-0.5) * qxx;
    meq[11] = qww;
    meq[12] = T(-0.5) * qww;
    meq[13] = q * jx * jy;
    meq[14] = q * jy * jz;
    meq[15] = q * jx * jz;
    meq[16] = meq[17] = meq[18] = T(0);
    const T uF = q * (jx * p.Fx + jy * p.Fy + jz * p.Fz);
    const T fxx = q * T(2) * (T(2) * jx * p.Fx - jy * p.Fy - jz * p.Fz);
    const T fww = q * T(2) * (jy * p.Fy - jz * p.Fz);
    mF[0] = T(0);
    mF[1] = T(38) * uF;
    mF[2] = T(-11) * uF;
    mF[3] = p.Fx;
    mF[4] = T(-2.0 / 3.0) * p.Fx;
    mF[5] = p.Fy;
    mF[6] = T(-2.0 / 3.0) * p.Fy;
    mF[7] = p.Fz;
    mF[8] = T(-2.0 / 3.0) * p.Fz;
    mF[9] = fxx;
    mF[10] = T(-0.5) * fxx;
    mF[11] = fww;
    mF[12] = T(-0.5) * fww;
    mF[13] = q * (jx * p.Fy + jy * p.Fx);
    mF[14] = q * (jy * p.Fz + jz * p.Fy);
    mF[15] = q * (jx * p.Fz + jz * p.Fx);
    mF[16] = mF[17] = mF[18] = T(0);
}

// g <- C(g), returning the shifted momentum j of the collided state.
template <typename T>
__device__ __forceinline__ void mrt_collide(T g[Q], const Collide<T> &p, T &jx_out, T &jy_out,
                                            T &jz_out) {
    T m[Q], meq[Q], mF[Q];
    moments_of<T>(g, m);
    const T jx = m[3] + T(0.5) * p.Fx, jy = m[5] + T(0.5) * p.Fy, jz = m[7] + T(0.5) * p.Fz;
    jx_out = jx;
    jy_out = jy;
    jz_out = jz;
    eq_and_force<T>(m[0], jx, jy, jz, p, meq, mF);
    // m*_k = m_k - s_k (m_k - meq_k) + (1 - s_k/2) mF_k, scaled by 1/D_k
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        const T s = rate_of<T>(k, p);
        m[k] = (m[k] - s * (m[k] - meq[k]) + (T(1) - T(0.5) * s) * mF[k]) * inv_norm<T>(k);
    }
    populations_from<T>(m, g);
}

}  // namespace lbm
