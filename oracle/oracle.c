/*
 * FP64 CPU oracle: D3Q19 MRT lattice Boltzmann with Guo forcing, halfway
 * bounceback and periodic boundaries, after Rao & Schaefer (arXiv:1902.11193).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline arm, never by the product library.  It shares no
 * code with the CUDA path.  Every operation is written out in its plainest
 * form: a dense 19x19 moment matrix M, its inverse M^T D^-1, the forcing
 * populations of eq. (Guo_Forcing) multiplied by M, and a two-array pull
 * stream.  OpenMP only splits independent z-planes; every sum is taken in a
 * fixed order, so results do not depend on the thread count.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 19
#define RHO0 1.0

/* D3Q19 velocity set (Sec. 2.1).  The paper names the lattice but prints no
 * ordering; rest first, then the six axis links, then the twelve edges. */
static const int CV[Q][3] = {
    {0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
    {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1}, {1, 0, -1},
    {-1, 0, 1}, {0, 1, 1},   {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

static double W[Q];
static int OPP[Q];
static double M[Q][Q];    /* m = M f */
static double MINV[Q][Q]; /* f = MINV m = M^T D^-1 m */
static int initialised = 0;

static void init_tables(void) {
    if (initialised) return;
    for (int i = 0; i < Q; ++i) {
        int c2 = CV[i][0] * CV[i][0] + CV[i][1] * CV[i][1] + CV[i][2] * CV[i][2];
        /* weights implied by eq. (BGK-EDF) with c_s^2 = 1/3 on D3Q19 */
        W[i] = c2 == 0 ? 1.0 / 3.0 : (c2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
        for (int j = 0; j < Q; ++j)
            if (CV[j][0] == -CV[i][0] && CV[j][1] == -CV[i][1] && CV[j][2] == -CV[i][2])
                OPP[i] = j;
    }
    /* Rows of M: the orthogonal polynomial basis of d'Humieres et al. (2002)
     * in the moment order of Sec. 2.2.1:
     * (rho, e, eps, jx, qx, jy, qy, jz, qz, 3pxx, 3pixx, pww, piww, pxy, pyz,
     *  pxz, mx, my, mz). */
    for (int i = 0; i < Q; ++i) {
        double x = CV[i][0], y = CV[i][1], z = CV[i][2];
        double c2 = x * x + y * y + z * z;
        M[0][i] = 1.0;
        M[1][i] = 19.0 * c2 - 30.0;
        M[2][i] = (21.0 * c2 * c2 - 53.0 * c2 + 24.0) / 2.0;
        M[3][i] = x;
        M[4][i] = (5.0 * c2 - 9.0) * x;
        M[5][i] = y;
        M[6][i] = (5.0 * c2 - 9.0) * y;
        M[7][i] = z;
        M[8][i] = (5.0 * c2 - 9.0) * z;
        M[9][i] = 3.0 * x * x - c2;
        M[10][i] = (3.0 * c2 - 5.0) * (3.0 * x * x - c2);
        M[11][i] = y * y - z * z;
        M[12][i] = (3.0 * c2 - 5.0) * (y * y - z * z);
        M[13][i] = x * y;
        M[14][i] = y * z;
        M[15][i] = x * z;
        M[16][i] = x * (y * y - z * z);
        M[17][i] = y * (z * z - x * x);
        M[18][i] = z * (x * x - y * y);
    }
    /* The rows are orthogonal, so M^-1 = M^T D^-1 with D = diag(M M^T). */
    for (int k = 0; k < Q; ++k) {
        double d = 0.0;
        for (int i = 0; i < Q; ++i) d += M[k][i] * M[k][i];
        for (int i = 0; i < Q; ++i) MINV[i][k] = M[k][i] / d;
    }
    initialised = 1;
}

void ora_lattice(int32_t c[Q * 3], double w[Q], int32_t opp[Q]) {
    init_tables();
    for (int i = 0; i < Q; ++i) {
        for (int a = 0; a < 3; ++a) c[3 * i + a] = CV[i][a];
        w[i] = W[i];
        opp[i] = OPP[i];
    }
}

void ora_moment_matrix(double Mout[Q * Q]) {
    init_tables();
    for (int k = 0; k < Q; ++k)
        for (int i = 0; i < Q; ++i) Mout[k * Q + i] = M[k][i];
}

/* Table 2.  s_nu = 1/tau in every set.  Kinetic rates:
 *   A: every other non-conserved rate 8(2 - s_nu)/(8 - s_nu)
 *   B: even rates s_nu; s_q = s_m = 8(2 - s_nu)/(8 - s_nu)
 *   C: s_e 1.19, s_eps 1.4, s_q 1.2, s_pi 1.4, s_m 1.98 (d'Humieres 2002)
 *   D: even rates s_nu; s_q = 8(2 - s_nu)/(8 - s_nu), s_m = 4(2 - s_nu)/(4 + s_nu)
 *   E: even rates s_nu; s_q = s_m = 2(2 - s_nu)/(4 Lambda s_nu - s_nu + 2),
 *      i.e. eq. (Magic param) held at Lambda
 *   SRT: every rate 1/tau (the BGK limit of Sec. 2.2.2). */
int ora_rates(int set, double tau, double Lambda, double s[Q]) {
    if (!(tau > 0.5)) return -1;
    double sn = 1.0 / tau;
    double se, seps, sq, spi, sm;
    double k8 = 8.0 * (2.0 - sn) / (8.0 - sn);
    switch (set) {
    case ORA_SET_A: se = seps = sq = spi = sm = k8; break;
    case ORA_SET_B: se = seps = spi = sn; sq = sm = k8; break;
    case ORA_SET_C: se = 1.19; seps = 1.4; sq = 1.2; spi = 1.4; sm = 1.98; break;
    case ORA_SET_D:
        se = seps = spi = sn;
        sq = k8;
        sm = 4.0 * (2.0 - sn) / (4.0 + sn);
        break;
    case ORA_SET_E:
        if (!(Lambda > 0.0)) return -1;
        se = seps = spi = sn;
        sq = sm = 2.0 * (2.0 - sn) / (4.0 * Lambda * sn - sn + 2.0);
        break;
    case ORA_SET_SRT: se = seps = sq = spi = sm = sn; break;
    default: return -1;
    }
    /* S = diag(0, se, seps, 0, sq, 0, sq, 0, sq, snu, spi, snu, spi, snu, snu,
     *          snu, sm, sm, sm), eq. (MRT params) */
    double t[Q] = {0.0, se, seps, 0.0, sq, 0.0, sq, 0.0, sq, sn,
                   spi, sn, spi, sn, sn, sn, sm, sm, sm};
    for (int k = 0; k < Q; ++k) s[k] = t[k];
    return 0;
}

/* eq. (MRT Equi) with rho0 = 1, read so that m^eq = M f^eq: m1 carries -11 rho
 * and m9 carries 2 jx^2 - jy^2 - jz^2 (the printed +11 rho and jx^2 - jy^2 -
 * jz^2 do not satisfy it), m10 = -m9/2, m12 = -m11/2.  With linear != 0 the
 * quadratic terms are dropped (the Stokes simplification of Sec. 2.2.1). */
void ora_meq(double rho, const double j[3], int linear, double meq[Q]) {
    double q = linear ? 0.0 : 1.0 / RHO0;
    double jx = j[0], jy = j[1], jz = j[2];
    double jj = jx * jx + jy * jy + jz * jz;
    meq[0] = rho;
    meq[1] = -11.0 * rho + 19.0 * q * jj;
    meq[2] = 3.0 * rho - 11.0 / 2.0 * q * jj;
    meq[3] = jx;
    meq[4] = -2.0 / 3.0 * jx;
    meq[5] = jy;
    meq[6] = -2.0 / 3.0 * jy;
    meq[7] = jz;
    meq[8] = -2.0 / 3.0 * jz;
    meq[9] = q * (2.0 * jx * jx - jy * jy - jz * jz);
    meq[10] = -0.5 * meq[9];
    meq[11] = q * (jy * jy - jz * jz);
    meq[12] = -0.5 * meq[11];
    meq[13] = q * jx * jy;
    meq[14] = q * jy * jz;
    meq[15] = q * jx * jz;
    meq[16] = meq[17] = meq[18] = 0.0;
}

/* eq. (Guo_Forcing) with c_s^2 = 1/3:
 * F_i = w_i [ (c_i - u)/c_s^2 + (c_i . u) c_i / c_s^4 ] . F.
 * linear != 0 drops the terms in u. */
void ora_guo_populations(const double u[3], const double F[3], int linear, double Fi[Q]) {
    init_tables();
    double ul[3] = {linear ? 0.0 : u[0], linear ? 0.0 : u[1], linear ? 0.0 : u[2]};
    for (int i = 0; i < Q; ++i) {
        double cu = CV[i][0] * ul[0] + CV[i][1] * ul[1] + CV[i][2] * ul[2];
        double acc = 0.0;
        for (int a = 0; a < 3; ++a)
            acc += (3.0 * (CV[i][a] - ul[a]) + 9.0 * cu * CV[i][a]) * F[a];
        Fi[i] = W[i] * acc;
    }
}

/* m^F = M . F_i: the paper computes the forcing populations first and then
 * multiplies by M (Sec. 2.2.1). */
void ora_force_moments(const double u[3], const double F[3], int linear, double mF[Q]) {
    double Fi[Q];
    ora_guo_populations(u, F, linear, Fi);
    for (int k = 0; k < Q; ++k) {
        double acc = 0.0;
        for (int i = 0; i < Q; ++i) acc += M[k][i] * Fi[i];
        mF[k] = acc;
    }
}

/* One node of eq. (MRT-LBE):
 *   m = M f;  rho = m0;  j = (m3, m5, m7) + F/2 (the shifted velocity of
 *   Sec. 2.2.1, rho0 u = sum_i c_i f_i + F/2);  u = j / rho0;
 *   m*_k = m_k - s_k (m_k - m^eq_k) + (1 - s_k/2) m^F_k;  f* = M^-1 m*. */
void ora_collide(const double f[Q], const double s[Q], const double F[3], int linear,
                 double fout[Q]) {
    init_tables();
    double m[Q], meq[Q], mF[Q], ms[Q];
    for (int k = 0; k < Q; ++k) {
        double acc = 0.0;
        for (int i = 0; i < Q; ++i) acc += M[k][i] * f[i];
        m[k] = acc;
    }
    double rho = m[0];
    double j[3] = {m[3] + 0.5 * F[0], m[5] + 0.5 * F[1], m[7] + 0.5 * F[2]};
    double u[3] = {j[0] / RHO0, j[1] / RHO0, j[2] / RHO0};
    ora_meq(rho, j, linear, meq);
    ora_force_moments(u, F, linear, mF);
    for (int k = 0; k < Q; ++k) ms[k] = m[k] - s[k] * (m[k] - meq[k]) + (1.0 - 0.5 * s[k]) * mF[k];
    for (int i = 0; i < Q; ++i) {
        double acc = 0.0;
        for (int k = 0; k < Q; ++k) acc += MINV[i][k] * ms[k];
        fout[i] = acc;
    }
}

/* Two-relaxation-time collision in link form (Sec. 2.2): each population is
 * split with its opposite into the symmetric half (f_i + f_opp)/2, relaxed
 * with s_plus, and the antisymmetric half (f_i - f_opp)/2, relaxed with
 * s_minus, towards the same halves of the second-order equilibrium
 * w_i [rho + 3 c.u + 9/2 (c.u)^2 - 3/2 u.u] (u = j/rho0, j shifted by F/2);
 * the Guo populations are split the same way and weighted (1 - s/2). */
void ora_trt_collide(const double f[Q], double s_plus, double s_minus, const double F[3],
                     int linear, double fout[Q]) {
    init_tables();
    double rho = 0.0, j[3] = {0.5 * F[0], 0.5 * F[1], 0.5 * F[2]};
    for (int i = 0; i < Q; ++i) {
        rho += f[i];
        for (int a = 0; a < 3; ++a) j[a] += CV[i][a] * f[i];
    }
    double u[3] = {j[0] / RHO0, j[1] / RHO0, j[2] / RHO0};
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    double feq[Q], Fi[Q];
    for (int i = 0; i < Q; ++i) {
        double cu = CV[i][0] * u[0] + CV[i][1] * u[1] + CV[i][2] * u[2];
        feq[i] = W[i] * (rho + 3.0 * cu + (linear ? 0.0 : 4.5 * cu * cu - 1.5 * uu));
    }
    ora_guo_populations(u, F, linear, Fi);
    for (int i = 0; i < Q; ++i) {
        int o = OPP[i];
        double fp = 0.5 * (f[i] + f[o]), fm = 0.5 * (f[i] - f[o]);
        double ep = 0.5 * (feq[i] + feq[o]), em = 0.5 * (feq[i] - feq[o]);
        double Fp = 0.5 * (Fi[i] + Fi[o]), Fm = 0.5 * (Fi[i] - Fi[o]);
        fout[i] = f[i] - s_plus * (fp - ep) - s_minus * (fm - em) + (1.0 - 0.5 * s_plus) * Fp +
                  (1.0 - 0.5 * s_minus) * Fm;
    }
}

static int wrapi(int v, int L) {
    int r = v % L;
    return r < 0 ? r + L : r;
}

int64_t ora_links(const uint8_t *mask, const int32_t dims[3], int32_t *fluid_idx,
                  int32_t *nbr, uint32_t *bbmask, int64_t links[Q]) {
    init_tables();
    int Lx = dims[0], Ly = dims[1], Lz = dims[2];
    int64_t N = (int64_t)Lx * Ly * Lz;
    int32_t *f_of_node = (int32_t *)malloc(sizeof(int32_t) * (size_t)(N > 0 ? N : 1));
    int64_t Nf = 0;
    for (int64_t n = 0; n < N; ++n) f_of_node[n] = mask[n] ? -1 : (int32_t)Nf++;
    if (links)
        for (int i = 0; i < Q; ++i) links[i] = 0;
    for (int z = 0; z < Lz; ++z)
        for (int y = 0; y < Ly; ++y)
            for (int x = 0; x < Lx; ++x) {
                int64_t n = x + (int64_t)Lx * (y + (int64_t)Ly * z);
                if (mask[n]) continue;
                int32_t fi = f_of_node[n];
                if (fluid_idx) fluid_idx[fi] = (int32_t)n;
                uint32_t bits = 0;
                for (int i = 1; i < Q; ++i) {
                    int xs = wrapi(x - CV[i][0], Lx), ys = wrapi(y - CV[i][1], Ly),
                        zs = wrapi(z - CV[i][2], Lz);
                    int64_t ns = xs + (int64_t)Lx * (ys + (int64_t)Ly * zs);
                    int32_t src = f_of_node[ns];
                    if (src < 0) {
                        bits |= 1u << i;
                        if (links) links[i]++;
                    }
                    if (nbr) nbr[(int64_t)(i - 1) * Nf + fi] = src;
                }
                if (bbmask) bbmask[fi] = bits;
            }
    free(f_of_node);
    return Nf;
}

struct ora_solver {
    int Lx, Ly, Lz;
    int64_t N;
    uint8_t *solid;
    double *f, *ftmp; /* [Q][N], post-collision state */
    double s[Q], F[3];
    int linear;
    int64_t steps;
    int fullway;   /* 0 halfway bounceback, 1 full-way bounceback */
    uint8_t *flag; /* full-way: 0 fluid, 1 bounceback voxel, 2 inner solid */
    int pressure_x;       /* x faces: Zou-He density boundaries instead of periodic */
    int symmetry;         /* bit 0: y faces, bit 1: z faces are symmetry (mirror) planes */
    double rho_in, rho_out;
};

/* Voxel flags of the paper's image analysis (Sec. 3), read with the mask as
 * the segmented image: a fluid voxel is flagged 0; a solid voxel with at
 * least one fluid voxel among its 18 link neighbours (periodic) is a
 * bounceback voxel, flag 1; any other solid voxel is flag 2. */
int64_t ora_flags(const uint8_t *mask, const int32_t dims[3], uint8_t *flags) {
    init_tables();
    const int Lx = dims[0], Ly = dims[1], Lz = dims[2];
    int64_t nbb = 0;
    for (int z = 0; z < Lz; ++z)
        for (int y = 0; y < Ly; ++y)
            for (int x = 0; x < Lx; ++x) {
                int64_t n = x + (int64_t)Lx * (y + (int64_t)Ly * z);
                uint8_t f = 0;
                if (mask[n]) {
                    f = 2;
                    for (int i = 1; i < Q; ++i) {
                        int64_t m = wrapi(x + CV[i][0], Lx) +
                                    (int64_t)Lx * (wrapi(y + CV[i][1], Ly) +
                                                   (int64_t)Ly * wrapi(z + CV[i][2], Lz));
                        if (!mask[m]) f = 1;
                    }
                }
                if (f == 1) ++nbb;
                flags[n] = f;
            }
    return nbb;
}

ora_solver *ora_create(const uint8_t *mask, const int32_t dims[3], const double s[Q],
                       const double F[3], int linear) {
    init_tables();
    if (dims[0] <= 0 || dims[1] <= 0 || dims[2] <= 0) return NULL;
    ora_solver *h = (ora_solver *)calloc(1, sizeof(ora_solver));
    h->Lx = dims[0];
    h->Ly = dims[1];
    h->Lz = dims[2];
    h->N = (int64_t)h->Lx * h->Ly * h->Lz;
    h->solid = (uint8_t *)malloc((size_t)h->N);
    memcpy(h->solid, mask, (size_t)h->N);
    h->f = (double *)malloc(sizeof(double) * Q * (size_t)h->N);
    h->ftmp = (double *)malloc(sizeof(double) * Q * (size_t)h->N);
    /* initial state: rest at rho0, f_i = w_i (the paper does not state one) */
    for (int i = 0; i < Q; ++i)
        for (int64_t n = 0; n < h->N; ++n) h->f[i * h->N + n] = W[i];
    for (int k = 0; k < Q; ++k) h->s[k] = s[k];
    for (int a = 0; a < 3; ++a) h->F[a] = F[a];
    h->linear = linear;
    return h;
}

int ora_set_bounceback(ora_solver *h, int mode) {
    if (!h || (mode != 0 && mode != 1)) return -1;
    if (mode == 1 && (h->pressure_x || h->symmetry)) return -1;
    h->fullway = mode;
    if (mode == 1 && !h->flag) {
        int32_t dims[3] = {h->Lx, h->Ly, h->Lz};
        h->flag = (uint8_t *)malloc((size_t)h->N);
        ora_flags(h->solid, dims, h->flag);
    }
    return 0;
}

void ora_destroy(ora_solver *h) {
    if (!h) return;
    free(h->flag);
    free(h->solid);
    free(h->f);
    free(h->ftmp);
    free(h);
}

/* Pull stream with halfway bounceback: f_i(x) = f*_i(x - c_i) when x - c_i
 * (periodic wrap) is fluid, else f*_opp(i)(x) (eq. LBE with the bounceback
 * rule applied at the half-link). */
static void pull(const ora_solver *h, const double *fs, int x, int y, int z, double fl[Q]) {
    int64_t n = x + (int64_t)h->Lx * (y + (int64_t)h->Ly * z);
    for (int i = 0; i < Q; ++i) {
        int xs = wrapi(x - CV[i][0], h->Lx), ys = wrapi(y - CV[i][1], h->Ly),
            zs = wrapi(z - CV[i][2], h->Lz);
        int64_t ns = xs + (int64_t)h->Lx * (ys + (int64_t)h->Ly * zs);
        fl[i] = h->solid[ns] ? fs[OPP[i] * h->N + n] : fs[i * h->N + ns];
    }
}

/* Pull stream without bounceback: f_i(x) = f*_i(x - c_i) from every
 * neighbour (full-way bounceback: the bounceback voxels hold populations). */
static void pull_all(const ora_solver *h, const double *fs, int x, int y, int z, double fl[Q]) {
    for (int i = 0; i < Q; ++i) {
        int xs = wrapi(x - CV[i][0], h->Lx), ys = wrapi(y - CV[i][1], h->Ly),
            zs = wrapi(z - CV[i][2], h->Lz);
        fl[i] = fs[i * h->N + xs + (int64_t)h->Lx * (ys + (int64_t)h->Ly * zs)];
    }
}

/* Direction with the y (axis 1) or z (axis 2) component of c_i reversed. */
static int mirror_dir(int i, int axis) {
    int c[3] = {CV[i][0], CV[i][1], CV[i][2]};
    c[axis] = -c[axis];
    for (int j = 0; j < Q; ++j)
        if (CV[j][0] == c[0] && CV[j][1] == c[1] && CV[j][2] == c[2]) return j;
    return -1;
}

/* Pull stream on a bounded domain (Sec. 2.4).
 * - y and/or z faces as symmetry planes (half a link outside the outer nodes):
 *   a population whose source lies outside is the specular image of the one
 *   that left the node next to it along the mirrored direction, so the
 *   source keeps the node's y (or z) and the direction's y (or z) component
 *   is reversed;
 * - x faces with prescribed density (Zou-He): populations entering through
 *   the face are unknown after streaming and are set by non-equilibrium
 *   bounceback, f_i = f_opp(i) + 6 w_i c_ix j_x - c_iy N_y - c_iz N_z, with
 *   j_x from the prescribed density and the known populations, and N_t half
 *   the tangential momentum of the in-plane populations, so that the node
 *   carries the prescribed density and no tangential momentum;
 * - halfway bounceback where the (mirrored) source voxel is solid. */
static void pull_bounded(const ora_solver *h, const double *fs, int x, int y, int z, double fl[Q]) {
    const int64_t n = x + (int64_t)h->Lx * (y + (int64_t)h->Ly * z);
    int unknown[Q] = {0}, any = 0;
    for (int i = 0; i < Q; ++i) {
        int xs = x - CV[i][0], ys = y - CV[i][1], zs = z - CV[i][2], dir = i;
        if (h->pressure_x && (xs < 0 || xs >= h->Lx)) {
            unknown[i] = any = 1;
            continue;
        }
        xs = wrapi(xs, h->Lx);
        if ((h->symmetry & 1) && (ys < 0 || ys >= h->Ly)) {
            ys = y;
            dir = mirror_dir(dir, 1);
        } else {
            ys = wrapi(ys, h->Ly);
        }
        if ((h->symmetry & 2) && (zs < 0 || zs >= h->Lz)) {
            zs = z;
            dir = mirror_dir(dir, 2);
        } else {
            zs = wrapi(zs, h->Lz);
        }
        int64_t ns = xs + (int64_t)h->Lx * (ys + (int64_t)h->Ly * zs);
        fl[i] = h->solid[ns] ? fs[OPP[i] * h->N + n] : fs[dir * h->N + ns];
    }
    if (!any) return;
    const int nx = (x == 0) ? 1 : -1; /* inward normal of the face */
    const double rho = (x == 0) ? h->rho_in : h->rho_out;
    double s0 = 0.0, sout = 0.0, Ny = 0.0, Nz = 0.0;
    for (int i = 0; i < Q; ++i) {
        if (CV[i][0] == 0) {
            s0 += fl[i];
            Ny += 0.5 * CV[i][1] * fl[i];
            Nz += 0.5 * CV[i][2] * fl[i];
        } else if (CV[i][0] == -nx) {
            sout += fl[i];
        }
    }
    const double jx = nx * (rho - s0 - 2.0 * sout);
    for (int i = 0; i < Q; ++i)
        if (unknown[i])
            fl[i] = fl[OPP[i]] + 6.0 * W[i] * CV[i][0] * jx - CV[i][1] * Ny - CV[i][2] * Nz;
}

int ora_set_domain(ora_solver *h, int pressure_x, double rho_in, double rho_out,
                   int symmetry) {
    if (!h || h->fullway || symmetry < 0 || symmetry > 3) return -1;
    if (pressure_x && (h->Lx < 2 || h->F[0] != 0.0 || h->F[1] != 0.0 || h->F[2] != 0.0 ||
                       !(rho_in > 0.0) || !(rho_out > 0.0)))
        return -1;
    h->pressure_x = pressure_x ? 1 : 0;
    h->symmetry = symmetry;
    h->rho_in = rho_in;
    h->rho_out = rho_out;
    return 0;
}

/* Velocity of a streamed node: u = (sum_i c_i f_i + F/2) / rho0. */
static void node_velocity(const ora_solver *h, const double fl[Q], double u[3]) {
    for (int a = 0; a < 3; ++a) {
        double acc = 0.0;
        for (int i = 0; i < Q; ++i) acc += CV[i][a] * fl[i];
        u[a] = (acc + 0.5 * h->F[a]) / RHO0;
    }
}

/* Sums per z-plane, then over planes in order: fixed summation order. */
static void one_step(ora_solver *h, double U[3]) {
    double *plane = U ? (double *)calloc(3 * (size_t)h->Lz, sizeof(double)) : NULL;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < h->Lz; ++z) {
        double fl[Q], fo[Q], u[3];
        for (int y = 0; y < h->Ly; ++y)
            for (int x = 0; x < h->Lx; ++x) {
                int64_t n = x + (int64_t)h->Lx * (y + (int64_t)h->Ly * z);
                if (h->fullway && h->flag[n] == 1) {
                    /* full-way bounceback: what streamed in goes back out
                     * along the opposite link in the next step */
                    pull_all(h, h->f, x, y, z, fl);
                    for (int i = 0; i < Q; ++i) h->ftmp[i * h->N + n] = fl[OPP[i]];
                    continue;
                }
                if (h->solid[n]) {
                    for (int i = 0; i < Q; ++i) h->ftmp[i * h->N + n] = h->f[i * h->N + n];
                    continue;
                }
                if (h->fullway)
                    pull_all(h, h->f, x, y, z, fl);
                else if (h->pressure_x || h->symmetry)
                    pull_bounded(h, h->f, x, y, z, fl);
                else
                    pull(h, h->f, x, y, z, fl);
                if (plane) {
                    node_velocity(h, fl, u);
                    for (int a = 0; a < 3; ++a) plane[3 * z + a] += u[a];
                }
                ora_collide(fl, h->s, h->F, h->linear, fo);
                for (int i = 0; i < Q; ++i) h->ftmp[i * h->N + n] = fo[i];
            }
    }
    double *t = h->f;
    h->f = h->ftmp;
    h->ftmp = t;
    h->steps++;
    if (U) {
        for (int a = 0; a < 3; ++a) {
            double acc = 0.0;
            for (int z = 0; z < h->Lz; ++z) acc += plane[3 * z + a];
            U[a] = acc / (double)h->N;
        }
        free(plane);
    }
}

void ora_step(ora_solver *h, int64_t n, double U[3]) {
    for (int64_t t = 0; t < n; ++t) one_step(h, t == n - 1 ? U : NULL);
}

void ora_velocity(ora_solver *h, double *u) {
#pragma omp parallel for schedule(static)
    for (int z = 0; z < h->Lz; ++z) {
        double fl[Q], v[3];
        for (int y = 0; y < h->Ly; ++y)
            for (int x = 0; x < h->Lx; ++x) {
                int64_t n = x + (int64_t)h->Lx * (y + (int64_t)h->Ly * z);
                if (h->solid[n]) {
                    for (int a = 0; a < 3; ++a) u[a * h->N + n] = 0.0;
                    continue;
                }
                if (h->fullway)
                    pull_all(h, h->f, x, y, z, fl);
                else if (h->pressure_x || h->symmetry)
                    pull_bounded(h, h->f, x, y, z, fl);
                else
                    pull(h, h->f, x, y, z, fl);
                node_velocity(h, fl, v);
                for (int a = 0; a < 3; ++a) u[a * h->N + n] = v[a];
            }
    }
}

void ora_mean_velocity(ora_solver *h, double U[3]) {
    double *u = (double *)malloc(sizeof(double) * 3 * (size_t)h->N);
    ora_velocity(h, u);
    for (int a = 0; a < 3; ++a) {
        double acc = 0.0;
        for (int z = 0; z < h->Lz; ++z) {
            double p = 0.0;
            for (int64_t r = 0; r < (int64_t)h->Lx * h->Ly; ++r)
                p += u[a * h->N + (int64_t)z * h->Lx * h->Ly + r];
            acc += p;
        }
        U[a] = acc / (double)h->N;
    }
    free(u);
}

void ora_get_f(ora_solver *h, double *f) { memcpy(f, h->f, sizeof(double) * Q * (size_t)h->N); }
void ora_set_f(ora_solver *h, const double *f) {
    memcpy(h->f, f, sizeof(double) * Q * (size_t)h->N);
}
int64_t ora_steps_done(ora_solver *h) { return h->steps; }

/* Stopping rule of eq. (convergence): the relative change of k (equivalently
 * of the mean velocity along the drive, k = nu U / F) between consecutive
 * steps.  It is evaluated on the last two steps of every chunk of K steps. */
int ora_run_to_convergence(ora_solver *h, double tol, int64_t K, int64_t max_steps,
                           int64_t *steps, double U[3]) {
    int d = 0;
    for (int a = 1; a < 3; ++a)
        if (fabs(h->F[a]) > fabs(h->F[d])) d = a;
    if (K < 1) K = 1;
    int64_t done = 0;
    double Ua[3] = {NAN, NAN, NAN}, Ub[3] = {NAN, NAN, NAN};
    int rc = 1;
    while (done < max_steps) {
        int64_t chunk = K;
        if (chunk > max_steps - done) chunk = max_steps - done;
        if (K == 1) {
            for (int a = 0; a < 3; ++a) Ua[a] = Ub[a];
            ora_step(h, 1, Ub);
        } else {
            if (chunk >= 2) ora_step(h, chunk - 2, NULL);
            if (chunk >= 2) ora_step(h, 1, Ua);
            else for (int a = 0; a < 3; ++a) Ua[a] = Ub[a];
            ora_step(h, 1, Ub);
        }
        done += chunk;
        if (!isfinite(Ub[0]) || !isfinite(Ub[1]) || !isfinite(Ub[2])) { rc = 2; break; }
        if (isfinite(Ua[d]) && fabs(Ub[d] - Ua[d]) <= tol * fabs(Ub[d])) { rc = 0; break; }
    }
    if (steps) *steps = done;
    if (U)
        for (int a = 0; a < 3; ++a) U[a] = Ub[a];
    return rc;
}

/* Rule 1 reads k^n of eq. (convergence) as the mean over steps n and n-1:
 * halfway bounceback in voxel gaps one or two voxels wide supports modes of
 * eigenvalue near -1 that make the per-step value alternate for tens of
 * thousands of steps around the fixed point; the two-step mean cancels them
 * and tends to the fixed point. */
int ora_run_to_convergence_rule(ora_solver *h, double tol, int64_t K, int64_t max_steps, int rule,
                                int64_t *steps, double U[3]) {
    if (rule == 0) return ora_run_to_convergence(h, tol, K, max_steps, steps, U);
    int d = 0;
    for (int a = 1; a < 3; ++a)
        if (fabs(h->F[a]) > fabs(h->F[d])) d = a;
    if (K < 3) K = 3;
    int64_t done = 0;
    double Ua[3], Ub[3], Uc[3], M[3] = {NAN, NAN, NAN};
    int rc = 1;
    while (done < max_steps) {
        int64_t chunk = K < max_steps - done ? K : max_steps - done;
        if (chunk < 3) {
            ora_step(h, chunk, NULL);
            done += chunk;
            break;
        }
        ora_step(h, chunk - 3, NULL);
        ora_step(h, 1, Ua);
        ora_step(h, 1, Ub);
        ora_step(h, 1, Uc);
        done += chunk;
        if (!isfinite(Uc[0]) || !isfinite(Uc[1]) || !isfinite(Uc[2])) {
            rc = 2;
            break;
        }
        double Ma[3];
        for (int a = 0; a < 3; ++a) {
            Ma[a] = 0.5 * (Ua[a] + Ub[a]);
            M[a] = 0.5 * (Ub[a] + Uc[a]);
        }
        if (fabs(M[d] - Ma[d]) <= tol * fabs(M[d])) {
            rc = 0;
            break;
        }
    }
    if (steps) *steps = done;
    if (U)
        for (int a = 0; a < 3; ++a) U[a] = M[a];
    return rc;
}

void ora_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int ora_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------- adjoint
 *
 * Not part of the paper: the sensitivity of the steady permeability to the
 * parameters (tau, the magic parameters, the force), written from the
 * definition of a fixed-point adjoint.  In the streamed variable h = S f*
 * one time step is h -> S C(h); at the steady state the adjoint psi solves
 * psi = J_C(h)^T S^T psi + dJ/dh with J = k along the drive, and
 * dk/dtheta = dJ/dtheta + (S^T psi) . dC/dtheta.  The collision C is a
 * quadratic polynomial in h and in F (and linear in each rate), so central
 * differences give its Jacobian and its F-derivative exactly up to rounding;
 * tau and Lambda enter through rational rate formulas and are differenced
 * with a small step. */

int ora_rates_magic(double tau, double Lq, double Lm, double s[Q]) {
    if (!(tau > 0.5) || !(Lq > 0.0) || !(Lm > 0.0)) return -1;
    double sn = 1.0 / tau;
    double sq = 2.0 * (2.0 - sn) / (4.0 * Lq * sn - sn + 2.0);
    double sm = 2.0 * (2.0 - sn) / (4.0 * Lm * sn - sn + 2.0);
    double t[Q] = {0.0, sn, sn, 0.0, sq, 0.0, sq, 0.0, sq, sn,
                   sn, sn, sn, sn, sn, sn, sm, sm, sm};
    for (int k = 0; k < Q; ++k) s[k] = t[k];
    return 0;
}

void ora_stream_field(ora_solver *h, const double *in, double *out) {
#pragma omp parallel for schedule(static)
    for (int z = 0; z < h->Lz; ++z) {
        double fl[Q];
        for (int y = 0; y < h->Ly; ++y)
            for (int x = 0; x < h->Lx; ++x) {
                int64_t n = x + (int64_t)h->Lx * (y + (int64_t)h->Ly * z);
                if (h->solid[n]) {
                    for (int i = 0; i < Q; ++i) out[i * h->N + n] = in[i * h->N + n];
                    continue;
                }
                pull(h, in, x, y, z, fl);
                for (int i = 0; i < Q; ++i) out[i * h->N + n] = fl[i];
            }
    }
}

/* (S^T v)(x, j): the post-collision population j of x streams to x + c_j
 * when that voxel is fluid, else it is bounced into slot opp(j) of x. */
static void unstream_node(const ora_solver *h, const double *v, int x, int y, int z,
                          double out[Q]) {
    int64_t n = x + (int64_t)h->Lx * (y + (int64_t)h->Ly * z);
    for (int j = 0; j < Q; ++j) {
        int xd = wrapi(x + CV[j][0], h->Lx), yd = wrapi(y + CV[j][1], h->Ly),
            zd = wrapi(z + CV[j][2], h->Lz);
        int64_t nd = xd + (int64_t)h->Lx * (yd + (int64_t)h->Ly * zd);
        out[j] = h->solid[nd] ? v[OPP[j] * h->N + n] : v[j * h->N + nd];
    }
}

void ora_unstream_field(ora_solver *h, const double *in, double *out) {
#pragma omp parallel for schedule(static)
    for (int z = 0; z < h->Lz; ++z) {
        double o[Q];
        for (int y = 0; y < h->Ly; ++y)
            for (int x = 0; x < h->Lx; ++x) {
                int64_t n = x + (int64_t)h->Lx * (y + (int64_t)h->Ly * z);
                if (h->solid[n]) {
                    for (int i = 0; i < Q; ++i) out[i * h->N + n] = in[i * h->N + n];
                    continue;
                }
                unstream_node(h, in, x, y, z, o);
                for (int i = 0; i < Q; ++i) out[i * h->N + n] = o[i];
            }
    }
}

/* Collision Jacobian J[i][c] = dC_i/dh_c at h: exact central differences
 * (C is quadratic in h). */
static void collide_jacobian(const double hs[Q], const double s[Q], const double F[3],
                             int linear, double J[Q][Q]) {
    const double d = 0.125;
    double hp[Q], hm[Q], cp[Q], cm[Q];
    for (int c = 0; c < Q; ++c) {
        for (int i = 0; i < Q; ++i) hp[i] = hm[i] = hs[i];
        hp[c] += d;
        hm[c] -= d;
        ora_collide(hp, s, F, linear, cp);
        ora_collide(hm, s, F, linear, cm);
        for (int i = 0; i < Q; ++i) J[i][c] = (cp[i] - cm[i]) / (2.0 * d);
    }
}

void ora_adjoint_apply(ora_solver *h, const double *in, double *out) {
    double *hs = (double *)malloc(sizeof(double) * Q * (size_t)h->N);
    ora_stream_field(h, h->f, hs);
#pragma omp parallel for schedule(static)
    for (int z = 0; z < h->Lz; ++z) {
        double hn[Q], phi[Q], J[Q][Q];
        for (int y = 0; y < h->Ly; ++y)
            for (int x = 0; x < h->Lx; ++x) {
                int64_t n = x + (int64_t)h->Lx * (y + (int64_t)h->Ly * z);
                if (h->solid[n]) {
                    for (int i = 0; i < Q; ++i) out[i * h->N + n] = 0.0;
                    continue;
                }
                for (int i = 0; i < Q; ++i) hn[i] = hs[i * h->N + n];
                collide_jacobian(hn, h->s, h->F, h->linear, J);
                unstream_node(h, in, x, y, z, phi);
                for (int c = 0; c < Q; ++c) {
                    double acc = 0.0;
                    for (int i = 0; i < Q; ++i) acc += J[i][c] * phi[i];
                    out[c * h->N + n] = acc;
                }
            }
    }
    free(hs);
}

/* Rates for a parameter point of the given set: p = {tau, Lambda, Lq, Lm};
 * the magic-parameter sets (B, D, E) are evaluated through Lq and Lm so that
 * they can be differentiated in each. */
static int rates_at(int set, const double p[4], double s[Q]) {
    if (set == ORA_SET_B || set == ORA_SET_D || set == ORA_SET_E)
        return ora_rates_magic(p[0], p[2], p[3], s);
    return ora_rates(set, p[0], p[1], s);
}

/* Adds to acc[0..6] one node's phi . dC/dtheta at the streamed populations
 * hn: theta = tau, Lambda (Set E), Lambda_q, Lambda_m (Sets B, D, E) by
 * central differences of the rates (step 1e-5), and the three force
 * components (C is quadratic in F, so the central difference is exact). */
static void node_param_grad(const ora_solver *h, int set, const double p0[4], int d,
                            const double hn[Q], const double phi[Q], double acc[7]) {
    double cp[Q], cm[Q], sp[Q], sm[Q];
    /* parameters 0..3: tau, Lambda, Lq, Lm */
    const double dp[4] = {1e-5, 1e-5, 1e-5, 1e-5};
    for (int q = 0; q < 4; ++q) {
        if (q == 1 && set != ORA_SET_E) continue;
        if ((q == 2 || q == 3) &&
            !(set == ORA_SET_B || set == ORA_SET_D || set == ORA_SET_E))
            continue;
        double pp[4], pm[4];
        for (int r = 0; r < 4; ++r) pp[r] = pm[r] = p0[r];
        if (q == 1) { /* Set E: Lambda moves both magic parameters */
            pp[2] += dp[1]; pp[3] += dp[1];
            pm[2] -= dp[1]; pm[3] -= dp[1];
        } else {
            pp[q] += dp[q];
            pm[q] -= dp[q];
        }
        rates_at(set, pp, sp);
        rates_at(set, pm, sm);
        ora_collide(hn, sp, h->F, h->linear, cp);
        ora_collide(hn, sm, h->F, h->linear, cm);
        double sum = 0.0;
        for (int i = 0; i < Q; ++i) sum += phi[i] * (cp[i] - cm[i]) / (2.0 * dp[q]);
        acc[q] += sum;
    }
    /* force components: C is quadratic in F */
    const double dF = 0.5 * fabs(h->F[d]);
    for (int a = 0; a < 3; ++a) {
        double Fp[3] = {h->F[0], h->F[1], h->F[2]}, Fm[3] = {h->F[0], h->F[1], h->F[2]};
        Fp[a] += dF;
        Fm[a] -= dF;
        ora_collide(hn, h->s, Fp, h->linear, cp);
        ora_collide(hn, h->s, Fm, h->linear, cm);
        double sum = 0.0;
        for (int i = 0; i < Q; ++i) sum += phi[i] * (cp[i] - cm[i]) / (2.0 * dF);
        acc[4 + a] += sum;
    }
}

int ora_adjoint(ora_solver *h, int set, double tau, double Lambda, double tol, int64_t K,
                int64_t max_iter, double grad[7], int64_t *iters) {
    init_tables();
    int d = 0;
    for (int a = 1; a < 3; ++a)
        if (fabs(h->F[a]) > fabs(h->F[d])) d = a;
    if (h->F[d] == 0.0 || h->fullway || h->pressure_x || h->symmetry) return -1;
    double p0[4] = {tau, Lambda, 3.0 / 16.0, 3.0 / 16.0};
    if (set == ORA_SET_D) p0[3] = 3.0 / 8.0;
    if (set == ORA_SET_E) p0[2] = p0[3] = Lambda;
    double s0[Q];
    if (rates_at(set, p0, s0) != 0) return -1;
    for (int k = 0; k < Q; ++k)
        if (fabs(s0[k] - h->s[k]) > 1e-14) return -1; /* rates must match the solver */
    if (K < 1) K = 1;

    const int64_t N = h->N;
    /* linearisation point: the mean of this step's and the next step's
     * streamed states (the solver advances one step) */
    double *hs = (double *)malloc(sizeof(double) * Q * (size_t)N);
    double *hs1 = (double *)malloc(sizeof(double) * Q * (size_t)N);
    ora_stream_field(h, h->f, hs);
    ora_step(h, 1, NULL);
    ora_stream_field(h, h->f, hs1);
    for (int64_t q = 0; q < (int64_t)Q * N; ++q) hs[q] = 0.5 * (hs[q] + hs1[q]);
    free(hs1);
    int64_t Nf = 0;
    for (int64_t n = 0; n < N; ++n) Nf += !h->solid[n];
    const double nu = (tau - 0.5) / 3.0;
    /* dJ/dh_i(x) = nu c_{i,d} / (F_d N) at fluid nodes, J = nu U_d / F_d */
    double *g = (double *)calloc((size_t)Q * N, sizeof(double));
    double *psi = (double *)calloc((size_t)Q * N, sizeof(double));
    double *nxt = (double *)calloc((size_t)Q * N, sizeof(double));
    double *old = (double *)calloc((size_t)Q * N, sizeof(double)); /* psi two iterations back */
    double Ud = 0.0;
    for (int64_t n = 0; n < N; ++n) {
        if (h->solid[n]) continue;
        double acc = 0.0;
        for (int i = 0; i < Q; ++i) {
            g[i * N + n] = nu * CV[i][d] / (h->F[d] * (double)N);
            acc += CV[i][d] * hs[i * N + n];
        }
        Ud += acc + 0.5 * h->F[d];
    }
    Ud /= (double)N;
    memcpy(psi, g, sizeof(double) * Q * (size_t)N);
    /* the steady state does not change: build every node's Jacobian once */
    double *Jac = (double *)malloc(sizeof(double) * Q * Q * (size_t)N);
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; ++n) {
        if (h->solid[n]) continue;
        double hn[Q];
        for (int i = 0; i < Q; ++i) hn[i] = hs[i * N + n];
        collide_jacobian(hn, h->s, h->F, h->linear, (double(*)[Q])(Jac + (size_t)n * Q * Q));
    }
    int rc = 1;
    int64_t it = 0;
    while (it < max_iter) {
        /* nxt = J_C^T S^T psi */
#pragma omp parallel for schedule(static)
        for (int z = 0; z < h->Lz; ++z) {
            double phi[Q];
            for (int y = 0; y < h->Ly; ++y)
                for (int x = 0; x < h->Lx; ++x) {
                    int64_t n = x + (int64_t)h->Lx * (y + (int64_t)h->Ly * z);
                    if (h->solid[n]) {
                        for (int i = 0; i < Q; ++i) nxt[i * N + n] = 0.0;
                        continue;
                    }
                    const double(*J)[Q] = (const double(*)[Q])(Jac + (size_t)n * Q * Q);
                    unstream_node(h, psi, x, y, z, phi);
                    for (int c = 0; c < Q; ++c) {
                        double acc = 0.0;
                        for (int i = 0; i < Q; ++i) acc += J[i][c] * phi[i];
                        nxt[c * N + n] = acc;
                    }
                }
        }
        /* change over two iterations: blind to a period-2 component */
        double dmax = 0.0, pmax = 0.0;
        for (int64_t q = 0; q < (int64_t)Q * N; ++q) {
            nxt[q] += g[q];
            double dd = fabs(nxt[q] - old[q]);
            if (dd > dmax) dmax = dd;
            if (fabs(nxt[q]) > pmax) pmax = fabs(nxt[q]);
        }
        double *t = old;
        old = psi;
        psi = nxt;
        nxt = t;
        ++it;
        if (it >= 2 && it % K == 0 && dmax <= tol * pmax) {
            rc = 0;
            break;
        }
    }
    /* the mean of the last two iterates */
    for (int64_t q = 0; q < (int64_t)Q * N; ++q) psi[q] = 0.5 * (psi[q] + old[q]);
    /* phi = S^T psi; gradient contributions per parameter */
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int z = 0; z < h->Lz; ++z)
        for (int y = 0; y < h->Ly; ++y)
            for (int x = 0; x < h->Lx; ++x) {
                int64_t n = x + (int64_t)h->Lx * (y + (int64_t)h->Ly * z);
                if (h->solid[n]) continue;
                double hn[Q], phi[Q];
                for (int i = 0; i < Q; ++i) hn[i] = hs[i * N + n];
                unstream_node(h, psi, x, y, z, phi);
                node_param_grad(h, set, p0, d, hn, phi, acc);
            }
    /* explicit dependence of J = nu(tau) U_d(h, F) / F_d on the parameters */
    grad[0] = acc[0] + Ud / (3.0 * h->F[d]);
    const int magic = set == ORA_SET_B || set == ORA_SET_D || set == ORA_SET_E;
    grad[1] = set == ORA_SET_E ? acc[1] : (magic ? acc[2] + acc[3] : NAN);
    grad[2] = magic ? acc[2] : NAN;
    grad[3] = magic ? acc[3] : NAN;
    for (int a = 0; a < 3; ++a) grad[4 + a] = acc[4 + a];
    grad[4 + d] += nu * ((double)Nf / (2.0 * (double)N)) / h->F[d] -
                   nu * Ud / (h->F[d] * h->F[d]);
    if (iters) *iters = it;
    free(Jac);
    free(hs);
    free(g);
    free(psi);
    free(nxt);
    free(old);
    return rc;
}

/* Gradient of the permeability after n more steps, J = nu U_d(S f_n) / F_d
 * with f_t the post-collision state t steps from now: reverse accumulation
 * through every step.  All n + 1 states are kept (the oracle runs small
 * lattices).  With h_t = S f_{t-1} the state step t collides,
 *   psi_{n+1} = dJ/dh,  psi_t = J_C(h_t)^T S^T psi_{t+1},
 *   dJ/dtheta = explicit + sum_t (S^T psi_{t+1}) . dC/dtheta(h_t). */
int ora_adjoint_transient(ora_solver *h, int set, double tau, double Lambda, int64_t n,
                          double grad[7]) {
    init_tables();
    int d = 0;
    for (int a = 1; a < 3; ++a)
        if (fabs(h->F[a]) > fabs(h->F[d])) d = a;
    if (n < 1 || h->F[d] == 0.0 || h->fullway || h->pressure_x || h->symmetry) return -1;
    double p0[4] = {tau, Lambda, 3.0 / 16.0, 3.0 / 16.0};
    if (set == ORA_SET_D) p0[3] = 3.0 / 8.0;
    if (set == ORA_SET_E) p0[2] = p0[3] = Lambda;
    double s0[Q];
    if (rates_at(set, p0, s0) != 0) return -1;
    for (int k = 0; k < Q; ++k)
        if (fabs(s0[k] - h->s[k]) > 1e-14) return -1;
    const int64_t N = h->N;
    const size_t field = (size_t)Q * N;
    double *fs = (double *)malloc(sizeof(double) * field * (size_t)(n + 1));
    if (!fs) return -1;
    memcpy(fs, h->f, sizeof(double) * field);
    for (int64_t t = 1; t <= n; ++t) {
        ora_step(h, 1, NULL);
        memcpy(fs + field * (size_t)t, h->f, sizeof(double) * field);
    }
    double *hs = (double *)malloc(sizeof(double) * field);
    double *psi = (double *)calloc(field, sizeof(double));
    double *nxt = (double *)calloc(field, sizeof(double));
    const double nu = (tau - 0.5) / 3.0;
    int64_t Nf = 0;
    double Ud = 0.0;
    ora_stream_field(h, fs + field * (size_t)n, hs);
    for (int64_t m = 0; m < N; ++m) {
        if (h->solid[m]) continue;
        ++Nf;
        double acc = 0.0;
        for (int i = 0; i < Q; ++i) {
            psi[i * N + m] = nu * CV[i][d] / (h->F[d] * (double)N);
            acc += CV[i][d] * hs[i * N + m];
        }
        Ud += acc + 0.5 * h->F[d];
    }
    Ud /= (double)N;
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int64_t t = n; t >= 1; --t) {
        ora_stream_field(h, fs + field * (size_t)(t - 1), hs); /* h_t */
        for (int z = 0; z < h->Lz; ++z)
            for (int y = 0; y < h->Ly; ++y)
                for (int x = 0; x < h->Lx; ++x) {
                    int64_t m = x + (int64_t)h->Lx * (y + (int64_t)h->Ly * z);
                    if (h->solid[m]) {
                        for (int i = 0; i < Q; ++i) nxt[i * N + m] = 0.0;
                        continue;
                    }
                    double hn[Q], phi[Q], J[Q][Q];
                    for (int i = 0; i < Q; ++i) hn[i] = hs[i * N + m];
                    unstream_node(h, psi, x, y, z, phi);
                    node_param_grad(h, set, p0, d, hn, phi, acc);
                    collide_jacobian(hn, h->s, h->F, h->linear, J);
                    for (int c = 0; c < Q; ++c) {
                        double v = 0.0;
                        for (int i = 0; i < Q; ++i) v += J[i][c] * phi[i];
                        nxt[c * N + m] = v;
                    }
                }
        double *tmp = psi;
        psi = nxt;
        nxt = tmp;
    }
    grad[0] = acc[0] + Ud / (3.0 * h->F[d]);
    const int magic = set == ORA_SET_B || set == ORA_SET_D || set == ORA_SET_E;
    grad[1] = set == ORA_SET_E ? acc[1] : (magic ? acc[2] + acc[3] : NAN);
    grad[2] = magic ? acc[2] : NAN;
    grad[3] = magic ? acc[3] : NAN;
    for (int a = 0; a < 3; ++a) grad[4 + a] = acc[4 + a];
    grad[4 + d] += nu * ((double)Nf / (2.0 * (double)N)) / h->F[d] -
                   nu * Ud / (h->F[d] * h->F[d]);
    free(fs);
    free(hs);
    free(psi);
    free(nxt);
    return 0;
}
