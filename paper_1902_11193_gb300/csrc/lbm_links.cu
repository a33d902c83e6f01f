// Link tables built on the device from the voxel mask (setup, once per
// lattice).
//
// Dense layouts keep one 32-bit link word per node: bit 31 = the voxel is
// solid, bit i (1..18) = the upstream neighbour x - c_i (periodic wrap) is
// solid, i.e. population i reaches x by halfway bounceback.  The paper's own
// pre-processing classifies voxels by their 18 neighbours (Sec. 3); this word
// is that classification per link, so the stream-collide kernel needs a
// single coalesced 4-byte load instead of 18 mask reads.
//
// The sparse layout lists fluid nodes in node order (fluid_idx), gives every
// fluid node the same bounceback bits (bb), and keeps per x-row fluid bit
// words with fluid-index bases (RowWord) and row starts, from which the
// stream-collide kernel computes upstream fluid indices (lbm_sparse.cuh).
// The explicit neighbour table nbr[18][Nf] (fluid index of x - c_i, -1 where
// solid) is only materialised on request, from the same computation.
// Per-direction bounceback link counts are accumulated with integer atomics,
// so they are exact.
#include "lbm_sparse.cuh"

namespace lbm {

__device__ __forceinline__ uint32_t upstream(uint32_t n, int j, int Lx, int Ly, int Lz) {
    uint32_t t = n / (uint32_t)Lx;
    int x = (int)(n - t * (uint32_t)Lx);
    int z = (int)(t / (uint32_t)Ly);
    int y = (int)(t - (uint32_t)z * (uint32_t)Ly);
    int xs = x - cx(j), ys = y - cy(j), zs = z - cz(j);
    xs = xs < 0 ? xs + Lx : (xs >= Lx ? xs - Lx : xs);
    ys = ys < 0 ? ys + Ly : (ys >= Ly ? ys - Ly : ys);
    zs = zs < 0 ? zs + Lz : (zs >= Lz ? zs - Lz : zs);
    return (uint32_t)xs + (uint32_t)Lx * ((uint32_t)ys + (uint32_t)Ly * (uint32_t)zs);
}

// Adds the block's count of each direction's bounceback flag to links[j]:
// warp popcounts into shared counters, then one global atomic per direction
// and block (all 18 directions of every warp hitting the same 18 global
// counters took 14 ms at 512^3).  Every thread of the block calls it.
__device__ __forceinline__ void count_links(uint32_t bits, bool valid,
                                            unsigned long long *links) {
    __shared__ unsigned cnt[Q];
    if (threadIdx.x < Q) cnt[threadIdx.x] = 0u;
    __syncthreads();
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 1; j < Q; ++j) {
        unsigned b = __ballot_sync(0xffffffffu, valid && (bits & (1u << j)));
        if (lane == 0 && b) atomicAdd(&cnt[j], (unsigned)__popc(b));
    }
    __syncthreads();
    if (threadIdx.x > 0 && threadIdx.x < Q && cnt[threadIdx.x])
        atomicAdd(links + threadIdx.x, (unsigned long long)cnt[threadIdx.x]);
}

// Dense link words.  Halfway mode: bounceback bits on fluid nodes, SOLID_BIT
// on solids.  Full-way mode: no bounceback bits (fluid nodes pull from every
// neighbour), BBNODE_BIT on solids with a fluid link neighbour, SOLID_BIT on
// the other solids.  The link counts are those of the mask in both modes.
__global__ void k_link_words(const uint8_t *__restrict__ mask, int Lx, int Ly, int Lz,
                             uint32_t N, int fullway, uint32_t *__restrict__ lw,
                             unsigned long long *links) {
    const uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t bits = 0;
    bool fluid = false;
    if (n < N) {
        uint32_t word;
        if (mask[n]) {
            word = SOLID_BIT;
            if (fullway) {
#pragma unroll
                for (int j = 1; j < Q; ++j)
                    if (!mask[upstream(n, j, Lx, Ly, Lz)]) word = BBNODE_BIT;
            }
        } else {
            fluid = true;
#pragma unroll
            for (int j = 1; j < Q; ++j)
                if (mask[upstream(n, j, Lx, Ly, Lz)]) bits |= 1u << j;
            word = fullway ? 0u : bits;
        }
        lw[n] = word;
    }
    count_links(bits, fluid, links);
}

// Fluid count per block of 1024 nodes.
__global__ void __launch_bounds__(1024) k_count_fluid(const uint8_t *__restrict__ mask, uint32_t N,
                                                      uint32_t *block_count) {
    const uint32_t n = blockIdx.x * 1024u + threadIdx.x;
    const bool f = n < N && mask[n] == 0;
    const unsigned b = __ballot_sync(0xffffffffu, f);
    __shared__ uint32_t sm[32];
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = __popc(b);
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t s = 0;
        for (int w = 0; w < 32; ++w) s += sm[w];
        block_count[blockIdx.x] = s;
    }
}

// Exclusive scan of the block counts by one block (setup only).
__global__ void __launch_bounds__(1024) k_scan_counts(const uint32_t *count, uint32_t nb,
                                                      uint32_t *offset, uint32_t *total) {
    __shared__ uint32_t sm[1024];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (uint32_t base = 0; base < nb; base += 1024) {
        const uint32_t i = base + threadIdx.x;
        const uint32_t v = i < nb ? count[i] : 0;
        sm[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {  // Hillis-Steele inclusive scan
            uint32_t t = threadIdx.x >= (unsigned)o ? sm[threadIdx.x - o] : 0;
            __syncthreads();
            sm[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < nb) offset[i] = carry + sm[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += sm[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

// Writes fluid_idx, the fluid-index base of every 32-voxel row word and the
// row starts.
__global__ void __launch_bounds__(1024) k_compact(const uint8_t *__restrict__ mask, uint32_t N,
                                                  const uint32_t *__restrict__ offset,
                                                  int32_t *fidx, int Lx,
                                                  int Wr, uint32_t nrows, RowWord *rw,
                                                  int32_t *rstart) {
    const uint32_t n = blockIdx.x * 1024u + threadIdx.x;
    const bool f = n < N && mask[n] == 0;
    const unsigned b = __ballot_sync(0xffffffffu, f);
    __shared__ uint32_t sm[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sm[wid] = __popc(b);
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t s = 0;
        for (int w = 0; w < 32; ++w) {
            uint32_t t = sm[w];
            sm[w] = s;
            s += t;
        }
    }
    __syncthreads();
    if (n < N) {
        // fluid nodes before n in node order = fluid index of n if fluid
        const uint32_t k = offset[blockIdx.x] + sm[wid] + __popc(b & ((1u << lane) - 1u));
        if (f) fidx[k] = (int32_t)n;
        const uint32_t R = n / (uint32_t)Lx;
        const uint32_t x = n - R * (uint32_t)Lx;
        if ((x & 31u) == 0) rw[(size_t)R * Wr + (x >> 5)].base = (int32_t)k;
        if (x == 0) rstart[R] = (int32_t)k;
        if (n == N - 1) rstart[nrows] = (int32_t)(k + (f ? 1u : 0u));
    }
}

// Fluid bits of every 32-voxel row word.
__global__ void k_row_bits(const uint8_t *__restrict__ mask, int Lx, int Wr, uint32_t nwords,
                           RowWord *rw) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nwords) return;
    const uint32_t R = t / (uint32_t)Wr, w = t - R * (uint32_t)Wr;
    uint32_t bits = 0;
    for (int b = 0; b < 32; ++b) {
        const int x = 32 * (int)w + b;
        if (x < Lx && mask[(size_t)x + (size_t)Lx * R] == 0) bits |= 1u << b;
    }
    rw[t].bits = bits;
}

// Materialises nbr[18][Nf] from the row map (fluid index of x - c_j, -1 if solid).
__global__ void k_sparse_nbr(SparseMap m, uint32_t Nf, int32_t *nbr) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= Nf) return;
    SparseNode sn;
    sn.init(k, m);
#pragma unroll
    for (int j = 1; j < Q; ++j)
        nbr[(size_t)(j - 1) * Nf + k] = (sn.bits & (1u << j)) ? -1 : (int32_t)sn.up(j, m);
}

__global__ void k_sparse_links(const int32_t *__restrict__ fidx, uint32_t Nf, int Lx, int Ly,
                               int Lz, const uint8_t *__restrict__ mask, uint32_t *bb,
                               uint2 *nb, unsigned long long *links) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t bits = 0;
    const bool valid = k < Nf;
    if (valid) {
        const uint32_t n = (uint32_t)fidx[k];
#pragma unroll
        for (int j = 1; j < Q; ++j) {
            if (mask[upstream(n, j, Lx, Ly, Lz)] != 0) bits |= 1u << j;
        }
        bb[k] = bits;
        nb[k] = make_uint2(n, bits);
    }
    count_links(bits, valid, links);
}

// Padded row tables of OddMap: row words and {row start, row end} of the
// lattice padded by one ghost row on each side in y and z.
__global__ void k_pad_rows(const RowWord *__restrict__ rw, const int32_t *__restrict__ rstart,
                           int Ly, int Lz, int Wr, uint32_t nwords, RowWord *rwp, int2 *rse) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nwords) return;
    const uint32_t p = t / (uint32_t)Wr, w = t - p * (uint32_t)Wr;
    const int yp = (int)(p % (uint32_t)(Ly + 2)), zp = (int)(p / (uint32_t)(Ly + 2));
    const int y = yp == 0 ? Ly - 1 : (yp == Ly + 1 ? 0 : yp - 1);
    const int z = zp == 0 ? Lz - 1 : (zp == Lz + 1 ? 0 : zp - 1);
    const uint32_t R = (uint32_t)y + (uint32_t)Ly * (uint32_t)z;
    rwp[t] = rw[(size_t)R * Wr + w];
    if (w == 0) rse[p] = make_int2(rstart[R], rstart[R + 1]);
}

// OddMap record of every fluid node: {padded row, bounceback bits | x << 19}.
__global__ void k_odd_records(const uint2 *__restrict__ nb, uint32_t Nf, int Lx, int Ly,
                              uint2 *orec) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= Nf) return;
    const uint2 v = nb[k];
    const uint32_t R = v.x / (uint32_t)Lx, x = v.x - R * (uint32_t)Lx;
    const uint32_t z = R / (uint32_t)Ly, y = R - z * (uint32_t)Ly;
    orec[k] = make_uint2((y + 1u) + (uint32_t)(Ly + 2) * (z + 1u), v.y | (x << 19));
}

// ---------------------------------------------------------------- launchers

int build_dense_links(lbm_ctx *c, unsigned long long *d_links) {
    const uint32_t N = (uint32_t)c->N;
    k_link_words<<<(N + 255) / 256, 256, 0, c->stream>>>(c->d_mask, c->Lx, c->Ly, c->Lz, N,
                                                          c->opt.bounceback, c->d_lw, d_links);
    c->launches++;
    return launch_error(cudaGetLastError());
}

int build_sparse_links(lbm_ctx *c, unsigned long long *d_links) {
    const uint32_t N = (uint32_t)c->N;
    const uint32_t nb = (N + 1023) / 1024;
    uint32_t *d_cnt = nullptr, *d_off = nullptr, *d_tot = nullptr;
    cudaError_t e = cudaMalloc(&d_cnt, sizeof(uint32_t) * (2 * (size_t)nb + 1));
    if (e != cudaSuccess) return launch_error(e);
    d_off = d_cnt + nb;
    d_tot = d_off + nb;
    k_count_fluid<<<nb, 1024, 0, c->stream>>>(c->d_mask, N, d_cnt);
    k_scan_counts<<<1, 1024, 0, c->stream>>>(d_cnt, nb, d_off, d_tot);
    const uint32_t nrows = (uint32_t)c->Ly * (uint32_t)c->Lz;
    const uint32_t nwords = nrows * (uint32_t)c->Wr;
    k_row_bits<<<(nwords + 255) / 256, 256, 0, c->stream>>>(c->d_mask, c->Lx, c->Wr, nwords, c->d_rw);
    k_compact<<<nb, 1024, 0, c->stream>>>(c->d_mask, N, d_off, c->d_fidx, c->Lx, c->Wr,
                                          nrows, c->d_rw, c->d_rstart);
    const uint32_t Nf = (uint32_t)c->Nf;
    if (Nf > 0)
        k_sparse_links<<<(Nf + 255) / 256, 256, 0, c->stream>>>(c->d_fidx, Nf, c->Lx, c->Ly, c->Lz,
                                                                 c->d_mask, c->d_bb, c->d_nb, d_links);
    c->launches += 5;
    if (c->d_orec) {
        const uint32_t pw = (uint32_t)(c->Ly + 2) * (uint32_t)(c->Lz + 2) * (uint32_t)c->Wr;
        k_pad_rows<<<(pw + 255) / 256, 256, 0, c->stream>>>(c->d_rw, c->d_rstart, c->Ly, c->Lz,
                                                            c->Wr, pw, c->d_rwp, c->d_rse);
        k_odd_records<<<(Nf + 255) / 256, 256, 0, c->stream>>>(c->d_nb, Nf, c->Lx, c->Ly,
                                                               c->d_orec);
        c->launches += 2;
    }
    uint32_t tot = 0;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&tot, d_tot, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d_cnt);
    if (e != cudaSuccess) return launch_error(e);
    if ((int64_t)tot != c->Nf) return LBM_ECUDA;
    return LBM_OK;
}

}  // namespace lbm

namespace lbm {
SparseMap sparse_map(const lbm_ctx *c);

int export_sparse_nbr(lbm_ctx *c, int32_t *nbr_dev) {
    const uint32_t Nf = (uint32_t)c->Nf;
    if (Nf == 0) return LBM_OK;
    k_sparse_nbr<<<(Nf + 255) / 256, 256, 0, c->stream>>>(sparse_map(c), Nf, nbr_dev);
    c->launches++;
    return launch_error(cudaGetLastError());
}
}  // namespace lbm
