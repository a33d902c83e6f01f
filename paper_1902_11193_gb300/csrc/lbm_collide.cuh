// The D3Q19 MRT collision with Guo forcing for one node, on shifted
// populations g_i = f_i - w_i (rho0 = 1).
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
#pragma once

#include "lbm_internal.cuh"

namespace lbm {

template <typename T>
__device__ __forceinline__ void mrt_collide(T g[Q], const Collide<T> &p, T &jx_out, T &jy_out,
                                            T &jz_out) {
    const T half = T(0.5);
    // opposite-pair sums (even part) and differences (odd part)
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

    // moments of the shifted populations
    const T rho = g[0] + sa + se;                         // m0 (deviation from rho0)
    const T e = T(-30) * g[0] - T(11) * sa + T(8) * se;   // m1
    const T eps = T(12) * g[0] - T(4) * sa + se;          // m2
    const T ex = d1 + d2 + d3 + d4;                       // edge part of x-odd moments
    const T ey = d1 - d2 + d5 + d6;
    const T ez = d3 - d4 + d5 - d6;
    const T jxr = dx + ex, qx = T(-4) * dx + ex;          // m3, m4
    const T jyr = dy + ey, qy = T(-4) * dy + ey;           // m5, m6
    const T jzr = dz + ez, qz = T(-4) * dz + ez;           // m7, m8
    const T pxx = T(2) * sx - sy - sz + sxy + sxz - T(2) * syz;       // m9
    const T pixx = T(-4) * sx + T(2) * (sy + sz) + sxy + sxz - T(2) * syz;  // m10
    const T pww = sy - sz + sxy - sxz;                      // m11
    const T piww = T(2) * (sz - sy) + sxy - sxz;            // m12
    const T pxy = s1 - s2;                                  // m13
    const T pyz = s5 - s6;                                  // m14
    const T pxz = s3 - s4;                                  // m15
    const T mx = d1 + d2 - d3 - d4;                         // m16
    const T my = d5 + d6 - d1 + d2;                         // m17
    const T mz = d3 - d4 - d5 + d6;                         // m18

    // shifted momentum j = sum c f + F/2 = rho0 u
    const T jx = jxr + half * p.Fx, jy = jyr + half * p.Fy, jz = jzr + half * p.Fz;
    jx_out = jx;
    jy_out = jy;
    jz_out = jz;

    // equilibrium (quadratic part) and forcing moments in u = j / rho0
    T jj = T(0), qxx = T(0), qww = T(0), qxy = T(0), qyz = T(0), qxz = T(0);
    T uF = T(0), fxx = T(0), fww = T(0), fxy = T(0), fyz = T(0), fxz = T(0);
    if (!p.linear) {
        jj = jx * jx + jy * jy + jz * jz;
        qxx = T(2) * jx * jx - jy * jy - jz * jz;
        qww = jy * jy - jz * jz;
        qxy = jx * jy;
        qyz = jy * jz;
        qxz = jx * jz;
        uF = jx * p.Fx + jy * p.Fy + jz * p.Fz;
        fxx = T(2) * (T(2) * jx * p.Fx - jy * p.Fy - jz * p.Fz);
        fww = T(2) * (jy * p.Fy - jz * p.Fz);
        fxy = jx * p.Fy + jy * p.Fx;
        fyz = jy * p.Fz + jz * p.Fy;
        fxz = jx * p.Fz + jz * p.Fx;
    }
    const T ke = T(1) - half * p.se, keps = T(1) - half * p.seps, kq = T(1) - half * p.sq;
    const T knu = T(1) - half * p.snu, kpi = T(1) - half * p.spi;

    // post-collision moments m*_k = m_k - s_k (m_k - meq_k) + (1 - s_k/2) mF_k
    const T e_s = e - p.se * (e - (T(-11) * rho + T(19) * jj)) + ke * (T(38) * uF);
    const T eps_s = eps - p.seps * (eps - (T(3) * rho - T(5.5) * jj)) + keps * (T(-11) * uF);
    const T twothird = T(2.0 / 3.0);
    const T qx_s = qx - p.sq * (qx + twothird * jx) - kq * twothird * p.Fx;
    const T qy_s = qy - p.sq * (qy + twothird * jy) - kq * twothird * p.Fy;
    const T qz_s = qz - p.sq * (qz + twothird * jz) - kq * twothird * p.Fz;
    const T jx_s = jxr + p.Fx, jy_s = jyr + p.Fy, jz_s = jzr + p.Fz;
    const T pxx_s = pxx - p.snu * (pxx - qxx) + knu * fxx;
    const T pixx_s = pixx - p.spi * (pixx + half * qxx) - kpi * half * fxx;
    const T pww_s = pww - p.snu * (pww - qww) + knu * fww;
    const T piww_s = piww - p.spi * (piww + half * qww) - kpi * half * fww;
    const T pxy_s = pxy - p.snu * (pxy - qxy) + knu * fxy;
    const T pyz_s = pyz - p.snu * (pyz - qyz) + knu * fyz;
    const T pxz_s = pxz - p.snu * (pxz - qxz) + knu * fxz;
    const T km = T(1) - p.sm;
    const T mx_s = km * mx, my_s = km * my, mz_s = km * mz;

    // f* = M^T D^-1 m*, with D = (19, 2394, 252, 10, 40, 10, 40, 10, 40, 36,
    // 72, 12, 24, 4, 4, 4, 8, 8, 8)
    const T a0 = rho * T(1.0 / 19.0);
    const T a1 = e_s * T(1.0 / 2394.0);
    const T a2 = eps_s * T(1.0 / 252.0);
    const T a3 = jx_s * T(0.1), a4 = qx_s * T(0.025);
    const T a5 = jy_s * T(0.1), a6 = qy_s * T(0.025);
    const T a7 = jz_s * T(0.1), a8 = qz_s * T(0.025);
    const T a9 = pxx_s * T(1.0 / 36.0), a10 = pixx_s * T(1.0 / 72.0);
    const T a11 = pww_s * T(1.0 / 12.0), a12 = piww_s * T(1.0 / 24.0);
    const T a13 = pxy_s * T(0.25), a14 = pyz_s * T(0.25), a15 = pxz_s * T(0.25);
    const T a16 = mx_s * T(0.125), a17 = my_s * T(0.125), a18 = mz_s * T(0.125);

    g[0] = a0 - T(30) * a1 + T(12) * a2;
    const T axis = a0 - T(11) * a1 - T(4) * a2;
    const T bx = axis + T(2) * a9 - T(4) * a10;
    const T ox = a3 - T(4) * a4;
    g[1] = bx + ox;
    g[2] = bx - ox;
    const T by = axis - a9 + T(2) * a10 + a11 - T(2) * a12;
    const T oy = a5 - T(4) * a6;
    g[3] = by + oy;
    g[4] = by - oy;
    const T bz = axis - a9 + T(2) * a10 - a11 + T(2) * a12;
    const T oz = a7 - T(4) * a8;
    g[5] = bz + oz;
    g[6] = bz - oz;

    const T edge = a0 + T(8) * a1 + a2;
    const T ox2 = a3 + a4, oy2 = a5 + a6, oz2 = a7 + a8;
    const T bxy = edge + a9 + a10 + a11 + a12;
    const T t1 = ox2 + oy2 + a16 - a17;
    g[7] = bxy + a13 + t1;
    g[8] = bxy + a13 - t1;
    const T t2 = ox2 - oy2 + a16 + a17;
    g[9] = bxy - a13 + t2;
    g[10] = bxy - a13 - t2;
    const T bxz = edge + a9 + a10 - a11 - a12;
    const T t3 = ox2 + oz2 - a16 + a18;
    g[11] = bxz + a15 + t3;
    g[12] = bxz + a15 - t3;
    const T t4 = ox2 - oz2 - a16 - a18;
    g[13] = bxz - a15 + t4;
    g[14] = bxz - a15 - t4;
    const T byz = edge - T(2) * (a9 + a10);
    const T t5 = oy2 + oz2 + a17 - a18;
    g[15] = byz + a14 + t5;
    g[16] = byz + a14 - t5;
    const T t6 = oy2 - oz2 + a17 + a18;
    g[17] = byz - a14 + t6;
    g[18] = byz - a14 - t6;
}

}  // namespace lbm
