/*
 * Seeded synthetic pore-space generators (binary voxel images).
 *
 * This file is the one input module shared by the FP64 CPU oracle's tests and
 * by the CUDA path: it only draws voxel masks and holds none of the lattice
 * Boltzmann arithmetic.  Masks are uint8 arrays laid out [Lz][Ly][Lx] with x
 * fastest; 1 = solid, 0 = fluid (the segmented image of Sec. 3, where the
 * paper's images come from micro-CT or drawn cross-sections).
 *
 * Voxelisation rule (the paper does not give one): voxel (i, j, k) is solid
 * iff its centre (i + 1/2, j + 1/2, k + 1/2) lies within distance <= r of a
 * sphere centre, measured with the periodic minimum image.
 *
 * Random centres come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), written here from its
 * published definition; a double in [0, 1) takes the top 53 bits.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GEOM_OK 0
#define GEOM_EINVAL (-1)

static uint64_t splitmix64_next(uint64_t *state) {
    uint64_t z = (*state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static double splitmix64_unit(uint64_t *state) {
    return (double)(splitmix64_next(state) >> 11) * (1.0 / 9007199254740992.0);
}

uint64_t geom_splitmix64(uint64_t *state) { return splitmix64_next(state); }

/* Signed periodic minimum-image offset of a - b on a ring of length L. */
static double min_image(double d, int L) {
    double h = 0.5 * (double)L;
    while (d >= h) d -= (double)L;
    while (d < -h) d += (double)L;
    return d;
}

static int wrap(long v, int L) {
    long r = v % (long)L;
    return (int)(r < 0 ? r + L : r);
}

/* Marks every voxel whose centre is within r of (cx, cy, cz); returns how many
 * voxels turned from fluid to solid. */
static int64_t paint_sphere(uint8_t *m, int Lx, int Ly, int Lz,
                            double cx, double cy, double cz, double r) {
    int64_t added = 0;
    double r2 = r * r;
    long x0 = (long)floor(cx - r - 1.0), x1 = (long)ceil(cx + r + 1.0);
    long y0 = (long)floor(cy - r - 1.0), y1 = (long)ceil(cy + r + 1.0);
    long z0 = (long)floor(cz - r - 1.0), z1 = (long)ceil(cz + r + 1.0);
    if (x1 - x0 + 1 >= Lx) { x0 = 0; x1 = Lx - 1; }
    if (y1 - y0 + 1 >= Ly) { y0 = 0; y1 = Ly - 1; }
    if (z1 - z0 + 1 >= Lz) { z0 = 0; z1 = Lz - 1; }
    for (long zz = z0; zz <= z1; ++zz) {
        int z = wrap(zz, Lz);
        double dz = min_image((double)z + 0.5 - cz, Lz);
        for (long yy = y0; yy <= y1; ++yy) {
            int y = wrap(yy, Ly);
            double dy = min_image((double)y + 0.5 - cy, Ly);
            double dyz = dy * dy + dz * dz;
            if (dyz > r2) continue;
            for (long xx = x0; xx <= x1; ++xx) {
                int x = wrap(xx, Lx);
                double dx = min_image((double)x + 0.5 - cx, Lx);
                if (dx * dx + dyz <= r2) {
                    size_t idx = (size_t)x + (size_t)Lx * ((size_t)y + (size_t)Ly * (size_t)z);
                    if (!m[idx]) { m[idx] = 1; ++added; }
                }
            }
        }
    }
    return added;
}

/* Periodic cubic unit cell of edge L holding one sphere array cell.
 * kind 0 = simple cubic (one sphere at the cell centre), 1 = body-centred
 * cubic (centre + corner), 2 = face-centred cubic (corner + three face
 * centres).  r is the sphere radius in voxels. */
int geom_sphere_array(uint8_t *mask, int L, int kind, double r) {
    if (!mask || L <= 0 || r < 0.0 || kind < 0 || kind > 2) return GEOM_EINVAL;
    size_t N = (size_t)L * L * L;
    memset(mask, 0, N);
    double h = 0.5 * (double)L;
    if (kind == 0) {
        paint_sphere(mask, L, L, L, h, h, h, r);
    } else if (kind == 1) {
        paint_sphere(mask, L, L, L, h, h, h, r);
        paint_sphere(mask, L, L, L, 0.0, 0.0, 0.0, r);
    } else {
        paint_sphere(mask, L, L, L, 0.0, 0.0, 0.0, r);
        paint_sphere(mask, L, L, L, h, h, 0.0, r);
        paint_sphere(mask, L, L, L, h, 0.0, h, r);
        paint_sphere(mask, L, L, L, 0.0, h, h, r);
    }
    return GEOM_OK;
}

/* Sphere radius that gives solid fraction c (before overlap) for n spheres
 * per cubic cell of edge L: c = n (4/3) pi r^3 / L^3. */
double geom_radius_for_fraction(int L, int spheres_per_cell, double c) {
    double V = (double)L * L * L;
    return cbrt(3.0 * c * V / (4.0 * M_PI * (double)spheres_per_cell));
}

/* Boolean (overlapping-sphere) medium: monodisperse spheres of radius r at
 * centres drawn uniformly in [0, L)^3 from SplitMix64(seed), added one by one
 * until the porosity is <= phi_target; the last sphere is kept.  Writes the
 * number of spheres and the final solid-voxel count. */
int geom_boolean(uint8_t *mask, int Lx, int Ly, int Lz, double r, double phi_target,
                 uint64_t seed, int64_t max_spheres, int64_t *n_spheres, int64_t *n_solid) {
    if (!mask || Lx <= 0 || Ly <= 0 || Lz <= 0 || r <= 0.0 || phi_target < 0.0 ||
        phi_target >= 1.0)
        return GEOM_EINVAL;
    size_t N = (size_t)Lx * Ly * Lz;
    memset(mask, 0, N);
    uint64_t st = seed;
    int64_t solid = 0, ns = 0;
    double target_solid = (1.0 - phi_target) * (double)N;
    while ((double)solid < target_solid && (max_spheres <= 0 || ns < max_spheres)) {
        double cx = splitmix64_unit(&st) * Lx;
        double cy = splitmix64_unit(&st) * Ly;
        double cz = splitmix64_unit(&st) * Lz;
        solid += paint_sphere(mask, Lx, Ly, Lz, cx, cy, cz, r);
        ++ns;
    }
    if (n_spheres) *n_spheres = ns;
    if (n_solid) *n_solid = solid;
    return GEOM_OK;
}

/* Union-find root with path halving. */
static int32_t uf_find(int32_t *p, int32_t a) {
    while (p[a] != a) {
        p[a] = p[p[a]];
        a = p[a];
    }
    return a;
}

/* Fills as solid every fluid cluster that is not the largest one, where two
 * fluid voxels belong to one cluster when a D3Q19 link (the 6 face and 12
 * edge neighbours, periodic wrap) joins them.  Enclosed pores carry no
 * steady flow; left in, a fully enclosed voxel under halfway bounceback keeps
 * a momentum mode that flips sign every step and never decays.  Returns the
 * number of voxels filled, or -1 on bad arguments / allocation failure. */
int64_t geom_fill_isolated(uint8_t *mask, int Lx, int Ly, int Lz) {
    if (!mask || Lx <= 0 || Ly <= 0 || Lz <= 0) return -1;
    const int64_t N = (int64_t)Lx * Ly * Lz;
    if (N >= ((int64_t)1 << 31)) return -1;
    int32_t *par = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    if (!par) return -1;
    for (int64_t n = 0; n < N; ++n) par[n] = (int32_t)n;
    /* half of the 18 links suffice: the other half are their opposites */
    static const int L9[9][3] = {{1, 0, 0},  {0, 1, 0}, {0, 0, 1},  {1, 1, 0}, {1, -1, 0},
                                 {1, 0, 1},  {1, 0, -1}, {0, 1, 1}, {0, 1, -1}};
    for (int z = 0; z < Lz; ++z)
        for (int y = 0; y < Ly; ++y)
            for (int x = 0; x < Lx; ++x) {
                const int64_t n = x + (int64_t)Lx * (y + (int64_t)Ly * z);
                if (mask[n]) continue;
                for (int k = 0; k < 9; ++k) {
                    const int xn = wrap((long)x + L9[k][0], Lx), yn = wrap((long)y + L9[k][1], Ly),
                              zn = wrap((long)z + L9[k][2], Lz);
                    const int64_t m = xn + (int64_t)Lx * (yn + (int64_t)Ly * zn);
                    if (mask[m]) continue;
                    const int32_t a = uf_find(par, (int32_t)n), b = uf_find(par, (int32_t)m);
                    if (a != b) par[a > b ? a : b] = a < b ? a : b;
                }
            }
    /* cluster sizes at the roots, then the largest */
    int32_t *size = (int32_t *)calloc((size_t)N, sizeof(int32_t));
    if (!size) {
        free(par);
        return -1;
    }
    int32_t best = -1, bestn = 0;
    for (int64_t n = 0; n < N; ++n) {
        if (mask[n]) continue;
        const int32_t r = uf_find(par, (int32_t)n);
        if (++size[r] > bestn || (size[r] == bestn && r < best)) {
            bestn = size[r];
            best = r;
        }
    }
    int64_t filled = 0;
    for (int64_t n = 0; n < N; ++n)
        if (!mask[n] && uf_find(par, (int32_t)n) != best) {
            mask[n] = 1;
            ++filled;
        }
    free(size);
    free(par);
    return filled;
}

/* Plane slit: H fluid layers (y = 0..H-1) and W solid layers (y = H..H+W-1),
 * uniform in x and z; lattice Lx x (H + W) x Lz. */
int geom_slit(uint8_t *mask, int Lx, int H, int W, int Lz) {
    if (!mask || Lx <= 0 || H <= 0 || W < 0 || Lz <= 0) return GEOM_EINVAL;
    int Ly = H + W;
    for (int z = 0; z < Lz; ++z)
        for (int y = 0; y < Ly; ++y)
            for (int x = 0; x < Lx; ++x)
                mask[(size_t)x + (size_t)Lx * ((size_t)y + (size_t)Ly * z)] = (uint8_t)(y >= H);
    return GEOM_OK;
}

/* Rectangular duct along x: fluid for 0 <= y < a and 0 <= z < b, one solid
 * layer at y = a and at z = b (periodic lattice Lx x (a+1) x (b+1)). */
int geom_duct(uint8_t *mask, int Lx, int a, int b) {
    if (!mask || Lx <= 0 || a <= 0 || b <= 0) return GEOM_EINVAL;
    int Ly = a + 1, Lz = b + 1;
    for (int z = 0; z < Lz; ++z)
        for (int y = 0; y < Ly; ++y)
            for (int x = 0; x < Lx; ++x)
                mask[(size_t)x + (size_t)Lx * ((size_t)y + (size_t)Ly * z)] =
                    (uint8_t)(y >= a || z >= b);
    return GEOM_OK;
}

/* Square block Lx x Ly x Lz with a circular bore of diameter D along x,
 * centred in the (y, z) cross-section: fluid iff the voxel centre is within
 * D/2 of the axis (the cylindrical channel of Sec. 4.1). */
int geom_pipe(uint8_t *mask, int Lx, int Ly, int Lz, double D) {
    if (!mask || Lx <= 0 || Ly <= 0 || Lz <= 0 || D <= 0.0) return GEOM_EINVAL;
    double R2 = 0.25 * D * D, cy = 0.5 * Ly, cz = 0.5 * Lz;
    for (int z = 0; z < Lz; ++z)
        for (int y = 0; y < Ly; ++y) {
            double dy = y + 0.5 - cy, dz = z + 0.5 - cz;
            uint8_t s = (uint8_t)(dy * dy + dz * dz > R2);
            for (int x = 0; x < Lx; ++x)
                mask[(size_t)x + (size_t)Lx * ((size_t)y + (size_t)Ly * z)] = s;
        }
    return GEOM_OK;
}

/* Equilateral triangular bore of side l along x, centred in the (y, z)
 * cross-section with one side parallel to y (the triangular channel of
 * Sec. 4.2): fluid iff the voxel centre is inside the triangle. */
int geom_triangle(uint8_t *mask, int Lx, int Ly, int Lz, double l) {
    if (!mask || Lx <= 0 || Ly <= 0 || Lz <= 0 || l <= 0.0) return GEOM_EINVAL;
    double h = l * sqrt(3.0) / 2.0;
    double cy = 0.5 * Ly, zb = 0.5 * Lz - h / 3.0; /* centroid at the centre */
    for (int z = 0; z < Lz; ++z)
        for (int y = 0; y < Ly; ++y) {
            double py = y + 0.5 - cy, pz = z + 0.5 - zb;
            /* inside iff above the base and below both slanted sides */
            int in = pz >= 0.0 && pz <= h && fabs(py) <= (h - pz) / sqrt(3.0);
            for (int x = 0; x < Lx; ++x)
                mask[(size_t)x + (size_t)Lx * ((size_t)y + (size_t)Ly * z)] = (uint8_t)!in;
        }
    return GEOM_OK;
}
