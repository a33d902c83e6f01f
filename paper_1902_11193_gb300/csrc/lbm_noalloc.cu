// Mean velocity of a caller-held FP64 population array without allocating
// device memory: a variant of the mean-velocity reduction (k_velocity +
// k_finalize) whose per-block partial sums live in a file-scope device
// array instead of memory the library allocates.
//
// Who needs it: callers that cannot call cudaMalloc at the point where they
// want the measurement, e.g. code embedded in a host application whose
// device memory is owned by another allocator (a framework's caching pool
// that must not be bypassed), or a loop that must not pay cudaMalloc's
// implicit device synchronisation.  They pass the populations, the mask and
// an output slot they already own; this file supplies the scratch.
//
// The lattice is read as the periodic, halfway-bounceback problem: any
// nonzero mask byte is a solid voxel, and a context built with full-way
// bounceback or bounded faces (pressure drive, symmetry planes) streams
// differently, so its mean velocity is not this call's.
//
// The scratch holds one partial sum per 256-node block, so the lattice is
// limited to LBM_NOALLOC_MAX_NODES nodes.  Every GPU that loads the library
// keeps the array (1.5 MiB) until the process exits.  All calls share it and
// it keeps the last call's contents; each call writes every slot it later
// reads, so nothing needs clearing, but two calls that overlap on the GPU
// (different streams, or different host threads on one device) race on it.
#include <math.h>
#include <string.h>

#include <mutex>

#include "lbm_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = LBM_NOALLOC_MAX_NODES / kThreads;

// partial sums (ux, uy, uz) per block
static __device__ __align__(256) double g_partials[3 * kMaxBlocks];

std::mutex g_mutex;
double *g_partials_addr[64] = {nullptr};  // device address of g_partials, per device

// Streamed-state velocity of the AB layout (post-collision populations f*
// of the last step, shifted by w): f_i(x) = f*_i(x - c_i), or f*_opp(i)(x)
// where x - c_i is solid (halfway bounceback); u = sum_i c_i f_i + F/2.
__global__ void __launch_bounds__(kThreads) k_velocity_static(const double *__restrict__ g,
                                                             const uint8_t *__restrict__ mask,
                                                             int Lx, int Ly, int Lz, double Fx,
                                                             double Fy, double Fz,
                                                             double *partials) {
    using namespace lbm;
    const uint32_t N = (uint32_t)Lx * Ly * Lz;
    const uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
    double v[3] = {0.0, 0.0, 0.0};
    if (n < N && !mask[n]) {
        const uint32_t t = n / (uint32_t)Lx;
        const int x = (int)(n - t * (uint32_t)Lx);
        const int z = (int)(t / (uint32_t)Ly);
        const int y = (int)(t - (uint32_t)z * (uint32_t)Ly);
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            int xs = x - cx(i), ys = y - cy(i), zs = z - cz(i);
            xs = xs < 0 ? xs + Lx : (xs >= Lx ? xs - Lx : xs);
            ys = ys < 0 ? ys + Ly : (ys >= Ly ? ys - Ly : ys);
            zs = zs < 0 ? zs + Lz : (zs >= Lz ? zs - Lz : zs);
            const uint32_t up = (uint32_t)xs + (uint32_t)Lx * ((uint32_t)ys + (uint32_t)Ly * (uint32_t)zs);
            // bounds-check build: an index out of range makes the result NaN
            // (this call has no context whose flag could carry it)
            if (kBoundsCheck && up >= N) {
                v[0] = v[1] = v[2] = NAN;
                break;
            }
            const double gi = mask[up] ? g[(size_t)opp(i) * N + n] : g[(size_t)i * N + up];
            v[0] += cx(i) * gi;
            v[1] += cy(i) * gi;
            v[2] += cz(i) * gi;
        }
        v[0] += 0.5 * Fx;
        v[1] += 0.5 * Fy;
        v[2] += 0.5 * Fz;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[a] += __shfl_down_sync(0xffffffffu, v[a], o);
    __shared__ double sm[kThreads / 32][3];
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int a = 0; a < 3; ++a) sm[threadIdx.x >> 5][a] = v[a];
    __syncthreads();
    if (threadIdx.x < 3) {
        double acc = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) acc += sm[w][threadIdx.x];
        partials[3 * (size_t)blockIdx.x + threadIdx.x] = acc;
    }
}

// Fixed-order sum of the partials: U[a] = sum / N.
__global__ void __launch_bounds__(1024) k_finalize_static(const double *__restrict__ partials,
                                                          int nblk, double inv_N, double *U) {
    __shared__ double sm[3][1024];
    double acc[3] = {0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblk; b += blockDim.x)
#pragma unroll
        for (int a = 0; a < 3; ++a) acc[a] += partials[3 * (size_t)b + a];
#pragma unroll
    for (int a = 0; a < 3; ++a) sm[a][threadIdx.x] = acc[a];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
#pragma unroll
            for (int a = 0; a < 3; ++a) sm[a][threadIdx.x] += sm[a][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < 3) U[threadIdx.x] = sm[threadIdx.x][0] * inv_N;
}

// Device address of the scratch array on the current device, looked up once
// per device (cudaGetSymbolAddress with that device current).
int scratch_address(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return lbm::launch_error(e);
    if (dev < 0 || dev >= 64) return LBM_EINVAL;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_partials_addr[dev]) {
        double *p = nullptr;
        e = cudaGetSymbolAddress((void **)&p, g_partials);
        if (e != cudaSuccess) return lbm::launch_error(e);
        g_partials_addr[dev] = p;
    }
    *out = g_partials_addr[dev];
    return LBM_OK;
}

}  // namespace

extern "C" int lbm_mean_velocity_noalloc(const double *f_dev, const uint8_t *mask_dev,
                                         const int32_t dims[3], const double force[3],
                                         double *U_dev, void *cuda_stream) {
    if (!f_dev || !mask_dev || !dims || !force || !U_dev) return LBM_EINVAL;
    if (dims[0] <= 0 || dims[1] <= 0 || dims[2] <= 0) return LBM_EINVAL;
    // each edge alone first, so that the product below cannot overflow
    const int64_t cap = LBM_NOALLOC_MAX_NODES;
    if (dims[0] > cap || dims[1] > cap || dims[2] > cap) return LBM_EINVAL;
    if ((int64_t)dims[0] * dims[1] > cap) return LBM_EINVAL;
    const int64_t N = (int64_t)dims[0] * dims[1] * dims[2];
    if (N > cap) return LBM_EINVAL;  // scratch holds N/256 partials
    double *partials = nullptr;
    int rc = scratch_address(&partials);
    if (rc != LBM_OK) return rc;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int nblk = (int)((N + kThreads - 1) / kThreads);
    k_velocity_static<<<nblk, kThreads, 0, s>>>(f_dev, mask_dev, dims[0], dims[1], dims[2],
                                                 force[0], force[1], force[2], partials);
    k_finalize_static<<<1, 1024, 0, s>>>(partials, nblk, 1.0 / (double)N, U_dev);
    return lbm::launch_error(cudaGetLastError());
}
