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

// Every add, multiply and fused multiply-add below is an explicitly rounded
// intrinsic (__fadd_rn, __fmul_rn, __fmaf_rn and their double forms).  The
// compiler may neither contract these into other FMAs nor reorder them, so
// every kernel that inlines the collision (single-lattice steps, the batched
// persistent kernel, the adjoint's state capture) performs the same
// roundings in the same order and produces the same bits for the same node.
// Left to itself the compiler fuses a*b + c where it sees fit, and that
// choice differs between kernels.
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float rsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float rfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double rsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double rfma(double a, double b, double c) { return __fma_rn(a, b, c); }

// m = M g.
template <typename T>
__device__ __forceinline__ void moments_of(const T g[Q], T m[Q]) {
    const T sx = radd(g[1], g[2]), dx = rsub(g[1], g[2]);
    const T sy = radd(g[3], g[4]), dy = rsub(g[3], g[4]);
    const T sz = radd(g[5], g[6]), dz = rsub(g[5], g[6]);
    const T s1 = radd(g[7], g[8]), d1 = rsub(g[7], g[8]);        // (1, 1, 0)
    const T s2 = radd(g[9], g[10]), d2 = rsub(g[9], g[10]);      // (1,-1, 0)
    const T s3 = radd(g[11], g[12]), d3 = rsub(g[11], g[12]);    // (1, 0, 1)
    const T s4 = radd(g[13], g[14]), d4 = rsub(g[13], g[14]);    // (1, 0,-1)
    const T s5 = radd(g[15], g[16]), d5 = rsub(g[15], g[16]);    // (0, 1, 1)
    const T s6 = radd(g[17], g[18]), d6 = rsub(g[17], g[18]);    // (0, 1,-1)
    const T syz_ax = radd(sy, sz);
    const T sa = radd(sx, syz_ax);
    const T sxy = radd(s1, s2), sxz = radd(s3, s4), syz = radd(s5, s6);
    const T sxy_xz = radd(sxy, sxz);
    const T se = radd(sxy_xz, syz);
    m[0] = radd(radd(g[0], sa), se);
    m[1] = rfma(T(-30), g[0], rfma(T(-11), sa, rmul(T(8), se)));
    m[2] = rfma(T(12), g[0], rfma(T(-4), sa, se));
    const T ex = radd(radd(d1, d2), radd(d3, d4));  // edge part of the x-odd moments
    const T ey = radd(rsub(d1, d2), radd(d5, d6));
    const T ez = radd(rsub(d3, d4), rsub(d5, d6));
    m[3] = radd(dx, ex);
    m[4] = rfma(T(-4), dx, ex);
    m[5] = radd(dy, ey);
    m[6] = rfma(T(-4), dy, ey);
    m[7] = radd(dz, ez);
    m[8] = rfma(T(-4), dz, ez);
    const T e9 = rfma(T(-2), syz, sxy_xz);  // sxy + sxz - 2 syz
    m[9] = rfma(T(2), sx, rsub(e9, syz_ax));
    m[10] = rfma(T(-4), sx, rfma(T(2), syz_ax, e9));
    const T dyz = rsub(sy, sz), dxyz = rsub(sxy, sxz);
    m[11] = radd(dyz, dxyz);
    m[12] = rfma(T(-2), dyz, dxyz);
    m[13] = rsub(s1, s2);
    m[14] = rsub(s5, s6);
    m[15] = rsub(s3, s4);
    m[16] = rsub(radd(d1, d2), radd(d3, d4));
    m[17] = rsub(radd(d5, d6), rsub(d1, d2));
    m[18] = rsub(rsub(d3, d4), rsub(d5, d6));
}

// g = M^T a (so g = M^-1 m for a_k = m_k / D_k).
template <typename T>
__device__ __forceinline__ void populations_from(const T a[Q], T g[Q]) {
    g[0] = rfma(T(12), a[2], rfma(T(-30), a[1], a[0]));
    const T axis = rfma(T(-4), a[2], rfma(T(-11), a[1], a[0]));
    const T bx = rfma(T(-4), a[10], rfma(T(2), a[9], axis));
    const T ox = rfma(T(-4), a[4], a[3]);
    g[1] = radd(bx, ox);
    g[2] = rsub(bx, ox);
    const T byz_ax = rfma(T(2), a[10], rsub(axis, a[9]));  // axis - a9 + 2 a10
    const T by = rfma(T(-2), a[12], radd(byz_ax, a[11]));
    const T oy = rfma(T(-4), a[6], a[5]);
    g[3] = radd(by, oy);
    g[4] = rsub(by, oy);
    const T bz = rfma(T(2), a[12], rsub(byz_ax, a[11]));
    const T oz = rfma(T(-4), a[8], a[7]);
    g[5] = radd(bz, oz);
    g[6] = rsub(bz, oz);
    const T edge = radd(rfma(T(8), a[1], a[0]), a[2]);
    const T ox2 = radd(a[3], a[4]), oy2 = radd(a[5], a[6]), oz2 = radd(a[7], a[8]);
    const T a910 = radd(a[9], a[10]), a1112 = radd(a[11], a[12]);
    const T e910 = radd(edge, a910);
    const T bxy = radd(e910, a1112);
    const T pxy = radd(bxy, a[13]), mxy = rsub(bxy, a[13]);
    const T t1 = radd(radd(ox2, oy2), rsub(a[16], a[17]));
    g[7] = radd(pxy, t1);
    g[8] = rsub(pxy, t1);
    const T t2 = radd(rsub(ox2, oy2), radd(a[16], a[17]));
    g[9] = radd(mxy, t2);
    g[10] = rsub(mxy, t2);
    const T bxz = rsub(e910, a1112);
    const T pxz = radd(bxz, a[15]), mxz = rsub(bxz, a[15]);
    const T t3 = radd(radd(ox2, oz2), rsub(a[18], a[16]));
    g[11] = radd(pxz, t3);
    g[12] = rsub(pxz, t3);
    const T t4 = rsub(rsub(ox2, oz2), radd(a[16], a[18]));
    g[13] = radd(mxz, t4);
    g[14] = rsub(mxz, t4);
    const T byz = rfma(T(-2), a910, edge);
    const T pyz = radd(byz, a[14]), myz = rsub(byz, a[14]);
    const T t5 = radd(radd(oy2, oz2), rsub(a[17], a[18]));
    g[15] = radd(pyz, t5);
    g[16] = rsub(pyz, t5);
    const T t6 = radd(rsub(oy2, oz2), radd(a[17], a[18]));
    g[17] = radd(myz, t6);
    g[18] = rsub(myz, t6);
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

// Forcing weight 1 - s_k/2 of moment k (non-conserved moments).
template <typename T>
__device__ __forceinline__ T half_of(int k, const Collide<T> &p) {
    return k == 1 ? p.he
         : k == 2 ? p.heps
         : (k == 4 || k == 6 || k == 8) ? p.hq
         : (k == 10 || k == 12) ? p.hpi
         : k >= 16 ? p.hm
                   : p.hnu;
}

// Equilibrium moments (shifted: rho is the deviation) and forcing moments
// for shifted momentum j (u = j / rho0, rho0 = 1).
template <typename T>
__device__ __forceinline__ void eq_and_force(T rho, T jx, T jy, T jz, const Collide<T> &p,
                                             T meq[Q], T mF[Q]) {
    const T q = p.q;
    const T q2 = rmul(T(2), p.q);
    const T xx = rmul(jx, jx), yy = rmul(jy, jy), zz = rmul(jz, jz);
    const T jj = rmul(q, radd(radd(xx, yy), zz));
    const T qxx = rmul(q, rsub(rsub(rmul(T(2), xx), yy), zz));
    const T qww = rmul(q, rsub(yy, zz));
    meq[0] = rho;
    meq[1] = rfma(T(19), jj, rmul(T(-11), rho));
    meq[2] = rfma(T(-5.5), jj, rmul(T(3), rho));
    meq[3] = jx;
    meq[4] = rmul(T(-2.0 / 3.0), jx);
    meq[5] = jy;
    meq[6] = rmul(T(-2.0 / 3.0), jy);
    meq[7] = jz;
    meq[8] = rmul(T(-2.0 / 3.0), jz);
    meq[9] = qxx;
    meq[10] = rmul(T(-0.5), qxx);
    meq[11] = qww;
    meq[12] = rmul(T(-0.5), qww);
    meq[13] = rmul(q, rmul(jx, jy));
    meq[14] = rmul(q, rmul(jy, jz));
    meq[15] = rmul(q, rmul(jx, jz));
    meq[16] = meq[17] = meq[18] = T(0);
    const T xF = rmul(jx, p.Fx), yF = rmul(jy, p.Fy), zF = rmul(jz, p.Fz);
    const T uF = rmul(q, radd(radd(xF, yF), zF));
    const T fxx = rmul(q2, rsub(rsub(rmul(T(2), xF), yF), zF));
    const T fww = rmul(q2, rsub(yF, zF));
    mF[0] = T(0);
    mF[1] = rmul(T(38), uF);
    mF[2] = rmul(T(-11), uF);
    mF[3] = p.Fx;
    mF[4] = rmul(T(-2.0 / 3.0), p.Fx);
    mF[5] = p.Fy;
    mF[6] = rmul(T(-2.0 / 3.0), p.Fy);
    mF[7] = p.Fz;
    mF[8] = rmul(T(-2.0 / 3.0), p.Fz);
    mF[9] = fxx;
    mF[10] = rmul(T(-0.5), fxx);
    mF[11] = fww;
    mF[12] = rmul(T(-0.5), fww);
    mF[13] = rmul(q, rfma(jx, p.Fy, rmul(jy, p.Fx)));
    mF[14] = rmul(q, rfma(jy, p.Fz, rmul(jz, p.Fy)));
    mF[15] = rmul(q, rfma(jx, p.Fz, rmul(jz, p.Fx)));
    mF[16] = mF[17] = mF[18] = T(0);
}

// g <- C(g), returning the shifted momentum j of the collided state.
template <typename T>
__device__ __forceinline__ void mrt_collide(T g[Q], const Collide<T> &p, T &jx_out, T &jy_out,
                                            T &jz_out) {
    T m[Q], meq[Q], mF[Q];
    moments_of<T>(g, m);
    const T jx = rfma(T(0.5), p.Fx, m[3]), jy = rfma(T(0.5), p.Fy, m[5]),
            jz = rfma(T(0.5), p.Fz, m[7]);
    jx_out = jx;
    jy_out = jy;
    jz_out = jz;
    eq_and_force<T>(m[0], jx, jy, jz, p, meq, mF);
    // m*_k = m_k - s_k (m_k - meq_k) + (1 - s_k/2) mF_k, scaled by 1/D_k.
    // The conserved moments (s_k = 0: rho, j) reduce to m_k + mF_k.
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        T r;
        if (k == 0 || k == 3 || k == 5 || k == 7) {
            r = k == 0 ? m[0] : radd(m[k], mF[k]);
        } else {
            const T s = rate_of<T>(k, p);
            r = rfma(-s, rsub(m[k], meq[k]), m[k]);
            r = rfma(half_of<T>(k, p), mF[k], r);
        }
        m[k] = rmul(r, inv_norm<T>(k));
    }
    populations_from<T>(m, g);
}

// Link-basis TRT collision (Sec. 2.2, the TRT model in link form).  For
// rates with a single even rate s+ (s_e = s_eps = s_nu = s_pi) and a single
// odd rate s- (s_q = s_m) -- Sets B and E and SRT -- the MRT collision above
// equals relaxing, for each opposite pair (i, opp(i)), the half sum
// S = (g_i + g_opp)/2 with s+ and the half difference D = (g_i - g_opp)/2
// with s- towards the same halves of the second-order equilibrium
// g_i^eq = w_i [rho + 3 c.u + 4.5 (c.u)^2 - 1.5 u.u] (shifted: rho is the
// deviation), with the Guo populations F_i = w_i [3 c.F - 3 u.F + 9 (c.u)(c.F)]
// split the same way and weighted (1 - s/2).  u = j + F/2 is the shifted
// momentum (rho0 = 1).  The conserved moments come out as in the MRT: the
// mass of (g - g^eq) and of F_i vanish, and the momentum row gives j + F.
// No moment transform, so fewer operations per node.

// c_i . (x, y, z) for the first direction i of a pair (odd i: its leading
// nonzero component is +1), rounded left to right.
template <typename T>
__device__ __forceinline__ T cdot_first(int i, T x, T y, T z) {
    T r = cx(i) != 0 ? x : (cy(i) != 0 ? y : z);
    if (cx(i) != 0 && cy(i) != 0) r = cy(i) > 0 ? radd(r, y) : rsub(r, y);
    if ((cx(i) != 0 || cy(i) != 0) && cz(i) != 0) r = cz(i) > 0 ? radd(r, z) : rsub(r, z);
    return r;
}

// sum over pairs k of sign(c_{2k+1, a}) d[k] for axis a, rounded in pair order
template <typename T>
__device__ __forceinline__ T pair_axis_sum(int a, const T d[9]) {
    T r = T(0);
    bool first = true;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const int i = 2 * k + 1;
        const int sg = a == 0 ? cx(i) : (a == 1 ? cy(i) : cz(i));
        if (sg == 0) continue;
        if (first) {
            r = sg > 0 ? d[k] : -d[k];
            first = false;
        } else {
            r = sg > 0 ? radd(r, d[k]) : rsub(r, d[k]);
        }
    }
    return r;
}

template <typename T>
__device__ __forceinline__ void trt_collide(T g[Q], const Collide<T> &p, T &jx_out, T &jy_out,
                                            T &jz_out) {
    const T q = p.q;
    const T sp = p.snu, sm = p.sq, hp = p.hnu, hm = p.hq;  // s+, s-, 1 - s+/2, 1 - s-/2
    T sum[9], dif[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        sum[k] = radd(g[2 * k + 1], g[2 * k + 2]);
        dif[k] = rsub(g[2 * k + 1], g[2 * k + 2]);
    }
    T rho = g[0];
#pragma unroll
    for (int k = 0; k < 9; ++k) rho = radd(rho, sum[k]);
    const T ux = rfma(T(0.5), p.Fx, pair_axis_sum<T>(0, dif));
    const T uy = rfma(T(0.5), p.Fy, pair_axis_sum<T>(1, dif));
    const T uz = rfma(T(0.5), p.Fz, pair_axis_sum<T>(2, dif));
    jx_out = ux;
    jy_out = uy;
    jz_out = uz;
    const T uu = rfma(uz, uz, rfma(uy, uy, rmul(ux, ux)));
    const T uF = rfma(uz, p.Fz, rfma(uy, p.Fy, rmul(ux, p.Fx)));
    const T A = rfma(rmul(T(-1.5), q), uu, rho);  // rho - 1.5 q u.u
    const T B = rmul(rmul(T(-3), q), uF);         // -3 q u.F
    const T q45 = rmul(T(4.5), q), q9 = rmul(T(9), q);
    {  // rest population: no antisymmetric half
        const T w0 = T(1.0 / 3.0);
        const T r = rfma(-sp, rsub(g[0], rmul(w0, A)), g[0]);
        g[0] = rfma(hp, rmul(w0, B), r);
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const int i = 2 * k + 1;
        const T w = T(weight(i));
        const T cu = cdot_first<T>(i, ux, uy, uz);
        const T cF = cdot_first<T>(i, p.Fx, p.Fy, p.Fz);
        const T Seq = rmul(w, rfma(rmul(q45, cu), cu, A));
        const T Fs = rmul(w, rfma(rmul(q9, cu), cF, B));
        const T Deq = rmul(T(3.0 * weight(i)), cu);
        const T Fd = rmul(T(3.0 * weight(i)), cF);
        const T S = rmul(T(0.5), sum[k]), D = rmul(T(0.5), dif[k]);
        const T Sn = rfma(hp, Fs, rfma(-sp, rsub(S, Seq), S));
        const T Dn = rfma(hm, Fd, rfma(-sm, rsub(D, Deq), D));
        g[i] = radd(Sn, Dn);
        g[i + 1] = rsub(Sn, Dn);
    }
}

// The collision a lattice uses: link-basis TRT where its rates allow it
// (p.trt), the moment-space MRT otherwise.  K fixes the choice at compile
// time (kCollideMrt, kCollideTrt): a kernel that carries both forms and
// branches between them runs a few per cent slower than either alone, so
// the single-lattice kernels are instantiated per form and the host picks
// one; kCollideRuntime branches on p.trt (the batched kernel, whose tiles
// belong to different lattices).
constexpr int kCollideRuntime = 0, kCollideMrt = 1, kCollideTrt = 2;

template <int K, typename T>
__device__ __forceinline__ void collide_as(T g[Q], const Collide<T> &p, T &jx_out, T &jy_out,
                                           T &jz_out) {
    if (K == kCollideTrt || (K == kCollideRuntime && p.trt))
        trt_collide<T>(g, p, jx_out, jy_out, jz_out);
    else
        mrt_collide<T>(g, p, jx_out, jy_out, jz_out);
}

}  // namespace lbm
