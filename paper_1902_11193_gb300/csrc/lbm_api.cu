// C ABI of liblbm_gb300 (declared in include/lbm.h): context life cycle,
// relaxation rates, time stepping, the stopping rule, permeability and the
// state readers/writers.  All device work is queued on the context stream.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <thread>
#include <vector>

#include "lbm_internal.cuh"

namespace lbm {
int launch_step(lbm_ctx *c, bool reduce);
int launch_velocity(lbm_ctx *c, double *u_dev, bool reduce);
int launch_step_bounded(lbm_ctx *c, bool reduce);
int launch_velocity_bounded(lbm_ctx *c, double *u_dev, bool reduce);
void launch_export(lbm_ctx *c, double *f_dev);
void launch_import(lbm_ctx *c, const double *f_dev);
void launch_export_at(lbm_ctx *c, const int64_t *nodes_dev, int count, double *f_dev);
void launch_finalize(lbm_ctx *c, int nblk, double inv_total, double *out_dev);
int build_dense_links(lbm_ctx *c, unsigned long long *d_links);
int build_sparse_links(lbm_ctx *c, unsigned long long *d_links);
int export_sparse_nbr(lbm_ctx *c, int32_t *nbr_dev);
int adjoint_sums(lbm_ctx *c, double tol, int64_t max_iter, int d, double coef, double sums[10],
                 int64_t *iters, double *resid);
int transient_sums(lbm_ctx *c, int64_t n, int d, double coef, double sums[10]);

static thread_local char g_cuda_err[256] = "";

int launch_error(cudaError_t e) {
    if (e == cudaSuccess) return LBM_OK;
    snprintf(g_cuda_err, sizeof g_cuda_err, "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA;
}
// The mask as uploaded at creation (the context keeps only the device copy).
static int host_mask(lbm_ctx *c, std::vector<uint8_t> &m) {
    m.resize((size_t)c->N);
    cudaError_t e = cudaMemcpyAsync(m.data(), c->d_mask, (size_t)c->N, cudaMemcpyDeviceToHost,
                                    c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return launch_error(e);
}
}  // namespace lbm

using namespace lbm;

#define CK(call)                                  \
    do {                                          \
        cudaError_t e_ = (call);                  \
        if (e_ != cudaSuccess) return launch_error(e_); \
    } while (0)

// Fluid count and value check of a host mask (every byte 0 or 1): eight
// bytes at a time (the set bits of 0/1 bytes are the solid voxels; any byte
// above 1 leaves a bit outside 0x01 in the OR of all words), split over up
// to 16 host threads for masks of 8 Mi voxels and more.  A 512^3 mask took
// 15 ms one byte at a time.
static void scan_range(const uint8_t *mask, int64_t b, int64_t e, uint64_t *acc_out,
                       int64_t *ones_out) {
    uint64_t acc = 0;
    int64_t ones = 0;
    int64_t n = b;
    for (; n + 8 <= e; n += 8) {
        uint64_t w;
        memcpy(&w, mask + n, 8);
        acc |= w;
        ones += __builtin_popcountll(w);
    }
    for (; n < e; ++n) {
        acc |= mask[n];
        ones += __builtin_popcountll(mask[n]);
    }
    *acc_out = acc;
    *ones_out = ones;
}

static bool scan_mask(const uint8_t *mask, int64_t N, int64_t *Nf) {
    constexpr int kMaxThreads = 16;
    const unsigned hw = std::thread::hardware_concurrency();
    int nt = (int)std::min<int64_t>(N >> 23, (int64_t)(hw > 0 ? hw : 1));
    nt = std::max(1, std::min(nt, kMaxThreads));
    uint64_t acc[kMaxThreads] = {};
    int64_t ones[kMaxThreads] = {};
    const int64_t per = ((N + nt - 1) / nt + 7) & ~int64_t(7);
    std::vector<std::thread> pool;
    pool.reserve(nt);  // no reallocation while threads are being started
    int started = 1;
    try {
        for (int t = 1; t < nt; ++t) {
            const int64_t b = std::min(N, t * per), e = std::min(N, b + per);
            pool.emplace_back(scan_range, mask, b, e, &acc[t], &ones[t]);
            ++started;
        }
    } catch (...) {  // no threads: the rest on this one
    }
    scan_range(mask, 0, std::min(N, per), &acc[0], &ones[0]);
    for (std::thread &th : pool) th.join();
    if (started < nt) {
        const int64_t b = std::min(N, started * per);
        scan_range(mask, b, N, &acc[started], &ones[started]);
        started = std::min(started + 1, nt);
    }
    uint64_t all = 0;
    int64_t solid = 0;
    for (int t = 0; t < started; ++t) {
        all |= acc[t];
        solid += ones[t];
    }
    if (all & 0xFEFEFEFEFEFEFEFEull) return false;
    *Nf = N - solid;
    return true;
}

extern "C" {

void lbm_default_options(lbm_options *o) {
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->precision = LBM_FP32_SHIFTED;
    o->layout = LBM_LAYOUT_AA;
    o->check_interval = 100;
    o->linear_eq = 0;
    o->max_steps = 1000000;
    o->cuda_stream = nullptr;
    o->fp16_scale_log2 = 0;
    o->block_size = 0;
    o->stop_rule = 0;
    o->bounceback = 0;
    o->pressure_x = 0;
    o->symmetry = 0;
    o->rho_in = 1.0;
    o->rho_out = 1.0;
    o->collision = 0;
    o->index_width = 0;
}

// Table 2 (Sec. 2.3); s_nu = 1/tau in every set.
int lbm_rates(int32_t set, double tau, double Lambda, double s[19]) {
    if (!s || !(tau > 0.5) || !isfinite(tau)) return LBM_EINVAL;
    const double sn = 1.0 / tau;
    const double k8 = 8.0 * (2.0 - sn) / (8.0 - sn);
    double se, seps, sq, spi, sm;
    switch (set) {
    case LBM_SET_A: se = seps = sq = spi = sm = k8; break;
    case LBM_SET_B: se = seps = spi = sn; sq = sm = k8; break;
    case LBM_SET_C: se = 1.19; seps = 1.4; sq = 1.2; spi = 1.4; sm = 1.98; break;
    case LBM_SET_D: se = seps = spi = sn; sq = k8; sm = 4.0 * (2.0 - sn) / (4.0 + sn); break;
    case LBM_SET_E:
        if (!(Lambda > 0.0) || !isfinite(Lambda)) return LBM_EINVAL;
        se = seps = spi = sn;
        sq = sm = 2.0 * (2.0 - sn) / (4.0 * Lambda * sn - sn + 2.0);
        break;
    case LBM_SET_SRT: se = seps = sq = spi = sm = sn; break;
    default: return LBM_EINVAL;
    }
    const double t[19] = {0, se, seps, 0, sq, 0, sq, 0, sq, sn, spi, sn, spi, sn, sn, sn, sm, sm, sm};
    memcpy(s, t, sizeof t);
    return LBM_OK;
}

static int check_rates(const double s[19]) {
    if (s[0] != 0.0 || s[3] != 0.0 || s[5] != 0.0 || s[7] != 0.0) return LBM_EINVAL;
    for (int k : {1, 2, 4, 9, 10, 16})
        if (!(s[k] > 0.0 && s[k] < 2.0)) return LBM_EINVAL;
    // the kernels use one rate per moment group of eq. (MRT params)
    if (s[6] != s[4] || s[8] != s[4] || s[11] != s[9] || s[13] != s[9] || s[14] != s[9] ||
        s[15] != s[9] || s[12] != s[10] || s[17] != s[16] || s[18] != s[16])
        return LBM_EINVAL;
    return LBM_OK;
}

static void free_ctx(lbm_ctx *c) {
    if (!c) return;
    cudaFree(c->d_mask);
    cudaFree(c->d_lw);
    cudaFree(c->d_fidx);
    cudaFree(c->d_bb);
    cudaFree(c->d_nb);
    cudaFree(c->d_rw);
    cudaFree(c->d_rstart);
    cudaFree(c->d_orec);
    cudaFree(c->d_rwp);
    cudaFree(c->d_rse);
    cudaFree(c->d_pop[0]);
    cudaFree(c->d_pop[1]);
    cudaFree(c->d_partials);
    cudaFree(c->d_U);
    cudaFree(c->d_flag);
    cudaFreeHost(c->h_U);
    for (int g = 0; g < kChunkGraphs; ++g)
        if (c->graphs[g].exec) cudaGraphExecDestroy(c->graphs[g].exec);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

// FP16 storage scale 2^S: puts the expected population deviation, of order
// the Stokes velocity |F| l^2 / (8 nu) for the mean pore chord l, near 2^12.
static int auto_fp16_scale(const lbm_ctx *c) {
    double Fm = fmax(fabs(c->F[0]), fmax(fabs(c->F[1]), fabs(c->F[2])));
    if (Fm <= 0.0) return 20;
    double faces = 0.0;
    for (int i = 1; i <= 6; ++i) faces += (double)c->links[i];
    const double phi = (double)c->Nf / (double)c->N;
    const double Sv = fmax(faces / (double)c->N * (2.0 / 3.0), 1e-12);
    double l = fmin(4.0 * phi / Sv, (double)fmax(c->Lx, fmax(c->Ly, c->Lz)));
    const double nu = (c->tau - 0.5) / 3.0;
    const double u = Fm * l * l / (8.0 * nu);
    int S = (int)floor(log2(4096.0 / fmax(u, 1e-30)));
    return S < 0 ? 0 : (S > 60 ? 60 : S);
}

int lbm_create_rates(lbm_ctx **out, const uint8_t *mask, const int32_t dims[3], const double s[19],
                     const double force[3], const lbm_options *opt) {
    if (!out || !mask || !dims || !s || !force) return LBM_EINVAL;
    *out = nullptr;
    if (dims[0] <= 0 || dims[1] <= 0 || dims[2] <= 0) return LBM_EINVAL;
    const int64_t N = (int64_t)dims[0] * dims[1] * dims[2];
    if (N >= (int64_t(1) << 31)) return LBM_EINVAL;
    if (check_rates(s) != LBM_OK) return LBM_EINVAL;
    for (int a = 0; a < 3; ++a)
        if (!isfinite(force[a])) return LBM_EINVAL;
    lbm_options o;
    lbm_default_options(&o);
    if (opt) o = *opt;
    if (o.block_size == 0) o.block_size = 256;
    if (o.block_size < 64 || o.block_size > 256 || (o.block_size & 31)) return LBM_EINVAL;
    if (o.precision < LBM_FP64 || o.precision > LBM_FP16_SHIFTED) return LBM_EINVAL;
    if (o.layout < LBM_LAYOUT_AB || o.layout > LBM_LAYOUT_SPARSE) return LBM_EINVAL;
    if (o.check_interval < 1) o.check_interval = 1;
    if (o.max_steps <= 0) o.max_steps = 1000000;
    if (o.fp16_scale_log2 < 0 || o.fp16_scale_log2 > 60) return LBM_EINVAL;
    if (o.stop_rule != 0 && o.stop_rule != 1) return LBM_EINVAL;
    if (o.bounceback != 0 && o.bounceback != 1) return LBM_EINVAL;
    if (o.bounceback == 1 && o.layout != LBM_LAYOUT_AB) return LBM_EINVAL;
    if ((o.pressure_x != 0 && o.pressure_x != 1) || o.symmetry < 0 || o.symmetry > 3)
        return LBM_EINVAL;
    if (o.collision != 0 && o.collision != 1) return LBM_EINVAL;
    if (o.index_width != 0 && o.index_width != 32 && o.index_width != 64) return LBM_EINVAL;
    if ((o.pressure_x || o.symmetry) && (o.layout != LBM_LAYOUT_AB || o.bounceback != 0))
        return LBM_EINVAL;
    if (o.pressure_x && (dims[0] < 2 || force[0] != 0.0 || force[1] != 0.0 || force[2] != 0.0 ||
                         !(o.rho_in > 0.0) || !(o.rho_out > 0.0) || !isfinite(o.rho_in) ||
                         !isfinite(o.rho_out)))
        return LBM_EINVAL;
    int64_t Nf = 0;
    if (!scan_mask(mask, N, &Nf)) return LBM_EINVAL;

    lbm_ctx *c = new (std::nothrow) lbm_ctx();
    if (!c) return LBM_ENOMEM;
    c->Lx = dims[0];
    c->Ly = dims[1];
    c->Lz = dims[2];
    c->N = N;
    c->Nf = Nf;
    memcpy(c->s, s, sizeof c->s);
    c->tau = 1.0 / s[9];
    memcpy(c->F, force, sizeof c->F);
    c->opt = o;
    c->set = -1;
    c->Lambda = NAN;
    c->converged = false;

    int rc = LBM_OK;
    auto fail = [&](int code) {
        free_ctx(c);
        return code;
    };
    cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) return fail(launch_error(e));
    if (o.cuda_stream) {
        c->stream = (cudaStream_t)o.cuda_stream;
        c->own_stream = false;
    } else {
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return fail(launch_error(e));
        c->own_stream = true;
    }
#define CKF(call)                                       \
    do {                                                \
        cudaError_t e2 = (call);                        \
        if (e2 != cudaSuccess) return fail(launch_error(e2)); \
    } while (0)
    CKF(cudaMalloc(&c->d_mask, (size_t)N));
    CKF(cudaMemcpyAsync(c->d_mask, mask, (size_t)N, cudaMemcpyHostToDevice, c->stream));
    unsigned long long *d_links = nullptr;
    CKF(cudaMalloc(&d_links, sizeof(unsigned long long) * 19));
    CKF(cudaMemsetAsync(d_links, 0, sizeof(unsigned long long) * 19, c->stream));
    const bool sparse = o.layout == LBM_LAYOUT_SPARSE;
    if (sparse) {
        CKF(cudaMalloc(&c->d_fidx, sizeof(int32_t) * (size_t)(Nf > 0 ? Nf : 1)));
        CKF(cudaMalloc(&c->d_bb, sizeof(uint32_t) * (size_t)(Nf > 0 ? Nf : 1)));
        CKF(cudaMalloc(&c->d_nb, sizeof(uint2) * (size_t)(Nf > 0 ? Nf : 1)));
        c->Wr = (c->Lx + 31) / 32;
        const size_t nrows = (size_t)c->Ly * c->Lz;
        CKF(cudaMalloc(&c->d_rw, sizeof(RowWord) * nrows * c->Wr));
        CKF(cudaMalloc(&c->d_rstart, sizeof(int32_t) * (nrows + 1)));
        if (Nf > 0 && (uint32_t)c->Lx < kOddMaxLx) {
            const size_t prows = (size_t)(c->Ly + 2) * (size_t)(c->Lz + 2);
            CKF(cudaMalloc(&c->d_orec, sizeof(uint2) * (size_t)Nf));
            CKF(cudaMalloc(&c->d_rwp, sizeof(RowWord) * prows * c->Wr));
            CKF(cudaMalloc(&c->d_rse, sizeof(int2) * prows));
        }
        rc = build_sparse_links(c, d_links);
    } else {
        CKF(cudaMalloc(&c->d_lw, sizeof(uint32_t) * (size_t)N));
        rc = build_dense_links(c, d_links);
    }
    if (rc != LBM_OK) {
        cudaFree(d_links);
        return fail(rc);
    }
    unsigned long long hl[19];
    CKF(cudaMemcpyAsync(hl, d_links, sizeof hl, cudaMemcpyDeviceToHost, c->stream));
    CKF(cudaStreamSynchronize(c->stream));
    cudaFree(d_links);
    for (int i = 0; i < 19; ++i) c->links[i] = (int64_t)hl[i];

    const int64_t units = sparse ? Nf : N;
    c->elem = o.precision == LBM_FP64 ? 8 : (o.precision == LBM_FP32_SHIFTED ? 4 : 2);
    const size_t bytes = c->elem * 19 * (size_t)(units > 0 ? units : 1);
    CKF(cudaMalloc(&c->d_pop[0], bytes));
    CKF(cudaMemsetAsync(c->d_pop[0], 0, bytes, c->stream));  // g = f - w = 0: rest state
    if (o.layout == LBM_LAYOUT_AB) {
        CKF(cudaMalloc(&c->d_pop[1], bytes));
        CKF(cudaMemsetAsync(c->d_pop[1], 0, bytes, c->stream));
    }
    // per-block partials for the largest grid a reducing launch can have
    c->n_partial_blocks = (int)((N + 63) / 64);
    CKF(cudaMalloc(&c->d_partials, sizeof(double) * 3 * (size_t)c->n_partial_blocks));
    CKF(cudaMalloc(&c->d_U, sizeof(double) * 24));
    CKF(cudaMalloc(&c->d_flag, sizeof(int)));
    CKF(cudaMemsetAsync(c->d_flag, 0, sizeof(int), c->stream));
    CKF(cudaMallocHost(&c->h_U, sizeof(double) * 26));
    if (o.precision == LBM_FP16_SHIFTED) {
        int S = o.fp16_scale_log2 ? o.fp16_scale_log2 : auto_fp16_scale(c);
        c->opt.fp16_scale_log2 = S;
        c->fp16_scale = ldexpf(1.0f, S);
    } else {
        c->fp16_scale = 0.0f;
    }
    CKF(cudaStreamSynchronize(c->stream));
#undef CKF
    *out = c;
    return LBM_OK;
}

int lbm_create(lbm_ctx **out, const uint8_t *mask, const int32_t dims[3], int32_t set, double tau,
               double Lambda, const double force[3], const lbm_options *opt) {
    double s[19];
    int rc = lbm_rates(set, tau, Lambda, s);
    if (rc != LBM_OK) return rc;
    rc = lbm_create_rates(out, mask, dims, s, force, opt);
    if (rc == LBM_OK) {
        (*out)->set = set;
        (*out)->Lambda = Lambda;
    }
    return rc;
}

void lbm_destroy(lbm_ctx *c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    free_ctx(c);
}

// Bounded domains (Zou-He faces, mirror planes) step and measure through
// their own kernels; everything else through the periodic ones.
static bool bounded(const lbm_ctx *c) { return c->opt.pressure_x || c->opt.symmetry; }
static int step_launch(lbm_ctx *c, bool reduce) {
    return bounded(c) ? launch_step_bounded(c, reduce) : launch_step(c, reduce);
}
static int velocity_launch(lbm_ctx *c, double *u_dev, bool reduce) {
    return bounded(c) ? launch_velocity_bounded(c, u_dev, reduce) : launch_velocity(c, u_dev, reduce);
}

// Drive of eq. (perm_calc) along axis a: the body force, or along x of a
// pressure-driven domain the pressure gradient c_s^2 (rho_in - rho_out)/(Lx - 1)
// between the face nodes.
static double drive_of(const lbm_ctx *c, int a) {
    if (c->opt.pressure_x)
        return a == 0 ? (c->opt.rho_in - c->opt.rho_out) / (3.0 * (double)(c->Lx - 1)) : 0.0;
    return c->F[a];
}

int lbm_step(lbm_ctx *c, int64_t n) {
    if (!c || n < 0) return LBM_EINVAL;
    if (n > 0) c->converged = c->has_conv = false;
    for (int64_t t = 0; t < n; ++t) step_launch(c, false);
    CK(cudaGetLastError());
    return LBM_OK;
}

// One measuring step: the mean streamed velocity lands in d_U[3*slot..].
static int measured_step(lbm_ctx *c, int slot) {
    int nblk = step_launch(c, true);
    if (nblk > 0)
        launch_finalize(c, nblk, 1.0 / (double)c->N, c->d_U + 3 * slot);
    else
        cudaMemsetAsync(c->d_U + 3 * slot, 0, 3 * sizeof(double), c->stream);
    return LBM_OK;
}

static void enqueue_chunk_direct(lbm_ctx *c, int64_t plain, int first, int nmeas) {
    for (int64_t t = 0; t < plain; ++t) step_launch(c, false);
    for (int m = 0; m < nmeas; ++m) measured_step(c, first + m);
}

// Longest chunk captured as a graph (launches); longer ones are enqueued
// directly, where launch overhead is negligible anyway.
constexpr int64_t kMaxGraphChunk = 4096;

// Enqueues `plain` plain steps, then measuring steps into slots first ..
// first + nmeas - 1.  A chunk of a given shape is captured once per context
// as a CUDA graph and replayed afterwards: on small lattices, where a step
// takes a few microseconds, the per-launch overhead otherwise dominates.
// Falls back to direct launches where the stream cannot be captured (it is
// being captured by the caller, or is the legacy default stream).
static int enqueue_chunk(lbm_ctx *c, int64_t plain, int first, int nmeas) {
    NvtxRange range("lbm chunk");
    const int phase = c->opt.layout == LBM_LAYOUT_AB ? c->cur : (int)(c->steps & 1);
    if (plain + nmeas < 2 || plain > kMaxGraphChunk) {
        enqueue_chunk_direct(c, plain, first, nmeas);
        return LBM_OK;
    }
    for (int g = 0; g < kChunkGraphs; ++g) {
        ChunkGraph &G = c->graphs[g];
        if (G.exec && G.plain == plain && G.first == first && G.nmeas == nmeas && G.phase == phase) {
            CK(cudaGraphLaunch(G.exec, c->stream));
            c->steps += plain + nmeas;
            c->launches += G.dlaunches;
            c->cur = G.cur_after;
            return LBM_OK;
        }
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(c->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone ||
        cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        enqueue_chunk_direct(c, plain, first, nmeas);
        return LBM_OK;
    }
    const int64_t steps0 = c->steps, launches0 = c->launches;
    const int cur0 = c->cur;
    enqueue_chunk_direct(c, plain, first, nmeas);
    const int64_t dlaunches = c->launches - launches0;
    const int cur_after = c->cur;
    c->steps = steps0;  // nothing ran yet: the capture only recorded the chunk
    c->launches = launches0;
    c->cur = cur0;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        cudaGetLastError();
        enqueue_chunk_direct(c, plain, first, nmeas);
        return LBM_OK;
    }
    ChunkGraph &G = c->graphs[c->next_graph];
    c->next_graph = (c->next_graph + 1) % kChunkGraphs;
    if (G.exec) cudaGraphExecDestroy(G.exec);
    G = ChunkGraph{exec, plain, first, nmeas, phase, dlaunches, cur_after};
    CK(cudaGraphLaunch(exec, c->stream));
    c->steps += plain + nmeas;
    c->launches += dlaunches;
    c->cur = cur_after;
    return LBM_OK;
}

static int read_U(lbm_ctx *c, int nslots) {
    CK(cudaMemcpyAsync(c->h_U, c->d_U, sizeof(double) * 3 * nslots, cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaMemcpyAsync((int *)(c->h_U + 24), c->d_flag, sizeof(int), cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

int lbm_run_to_convergence(lbm_ctx *c, double tol, int64_t *steps_taken) {
    if (!c || !(tol >= 0.0)) return LBM_EINVAL;
    int d = 0;
    for (int a = 1; a < 3; ++a)
        if (fabs(drive_of(c, a)) > fabs(drive_of(c, d))) d = a;
    const int rule = c->opt.stop_rule;
    const int64_t K = rule == 1 && c->opt.check_interval < 3 ? 3 : c->opt.check_interval;
    const int64_t maxs = c->opt.max_steps;
    int64_t done = 0;
    c->converged = false;
    c->has_conv = false;
    double Ua = NAN, Ub = NAN;
    double Uc3[3] = {NAN, NAN, NAN};
    int rc = LBM_ENOTCONV;
    c->history.clear();
    NvtxRange range("lbm_run_to_convergence");
    auto note = [&]() {
        lbm_check r;
        r.step = c->steps;
        r.U = Ub;
        r.change = isfinite(Ua) ? fabs(Ub - Ua) / fabs(Ub) : NAN;
        c->history.push_back(r);
    };
    while (done < maxs) {
        int64_t chunk = K < maxs - done ? K : maxs - done;
        int rr;
        if (rule == 1) {
            // the mean of two consecutive steps, from the chunk's last three
            if (chunk < 3) {
                for (int64_t t = 0; t < chunk; ++t) step_launch(c, false);
                CK(cudaGetLastError());
                done += chunk;
                break;
            }
            rr = enqueue_chunk(c, chunk - 3, 0, 3);
            if (rr) return rr;
            CK(cudaGetLastError());
            rr = read_U(c, 3);
            if (rr) return rr;
            for (int a = 0; a < 3; ++a) Uc3[a] = 0.5 * (c->h_U[3 + a] + c->h_U[6 + a]);
            Ua = 0.5 * (c->h_U[d] + c->h_U[3 + d]);
            Ub = Uc3[d];
            done += chunk;
            note();
            const int flag = *(int *)(c->h_U + 24);
            if (flag || !isfinite(c->h_U[6]) || !isfinite(c->h_U[7]) || !isfinite(c->h_U[8])) {
                rc = LBM_EUNSTABLE;
                break;
            }
            if (fabs(Ub - Ua) <= tol * fabs(Ub)) {
                rc = LBM_OK;
                break;
            }
            continue;
        }
        if (K >= 2 && chunk >= 2) {
            rr = enqueue_chunk(c, chunk - 2, 0, 2);
            if (rr) return rr;
            CK(cudaGetLastError());
            rr = read_U(c, 2);
            if (rr) return rr;
            Ua = c->h_U[d];
            Ub = c->h_U[3 + d];
        } else {
            measured_step(c, 1);
            CK(cudaGetLastError());
            rr = read_U(c, 2);
            if (rr) return rr;
            Ua = Ub;
            Ub = c->h_U[3 + d];
        }
        done += chunk;
        note();
        const int flag = *(int *)(c->h_U + 24);
        if (flag || !isfinite(c->h_U[3]) || !isfinite(c->h_U[4]) || !isfinite(c->h_U[5])) {
            rc = LBM_EUNSTABLE;
            break;
        }
        for (int a = 0; a < 3; ++a) Uc3[a] = c->h_U[3 + a];
        if (isfinite(Ua) && fabs(Ub - Ua) <= tol * fabs(Ub)) {
            rc = LBM_OK;
            break;
        }
    }
    if (steps_taken) *steps_taken = done;
    c->converged = rc == LBM_OK;
    if (rc == LBM_OK || rc == LBM_ENOTCONV) {
        c->has_conv = isfinite(Uc3[0]);
        for (int a = 0; a < 3; ++a) c->U_conv[a] = Uc3[a];
    }
    return rc;
}

int lbm_convergence_history(lbm_ctx *c, lbm_check *out, int64_t cap, int64_t *count) {
    if (!c || cap < 0) return LBM_EINVAL;
    const int64_t n = (int64_t)c->history.size();
    if (out)
        for (int64_t i = 0; i < n && i < cap; ++i) out[i] = c->history[(size_t)i];
    if (count) *count = n;
    return LBM_OK;
}

int lbm_device_flags(lbm_ctx *c, int32_t *flags) {
    if (!c || !flags) return LBM_EINVAL;
    int h = 0;
    CK(cudaMemcpyAsync(&h, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemsetAsync(c->d_flag, 0, sizeof(int), c->stream));
    CK(cudaStreamSynchronize(c->stream));
    *flags = h;
    return LBM_OK;
}

int lbm_converged_velocity(lbm_ctx *c, double U[3]) {
    if (!c || !U) return LBM_EINVAL;
    if (!c->has_conv) return LBM_ENOSTATE;
    for (int a = 0; a < 3; ++a) U[a] = c->U_conv[a];
    return LBM_OK;
}

int lbm_converged_permeability(lbm_ctx *c, double k[3]) {
    if (!c || !k) return LBM_EINVAL;
    if (!c->has_conv) return LBM_ENOSTATE;
    const double nu = (c->tau - 0.5) / 3.0;
    for (int a = 0; a < 3; ++a) {
        const double g = drive_of(c, a);
        k[a] = g != 0.0 ? nu * c->U_conv[a] / g : NAN;
    }
    return LBM_OK;
}

// d s_E / d s_nu and d s_E / d Lambda for s_E = 2(2 - s)/(4 Lambda s - s + 2)
// (eq. Magic param solved for the odd rate).
static double dsE_ds(double s, double L) {
    const double den = 4.0 * L * s - s + 2.0;
    return -16.0 * L / (den * den);
}
static double dsE_dL(double s, double L) {
    const double den = 4.0 * L * s - s + 2.0;
    return -8.0 * s * (2.0 - s) / (den * den);
}

// The chain rule from the raw gradient sums (see k_adj_grad) to lbm_grad:
// through Table 2's rate rules for the set, plus the explicit dependence of
// J = nu(tau) U_d / F_d on tau and F.
static void fill_grad(lbm_ctx *c, int d, const double sums[10], int64_t iters, double resid,
                      lbm_grad *out) {
    const double tau = c->tau, sn = c->s[9], nu = (tau - 0.5) / 3.0, Fd = c->F[d];
    const double Nd = (double)c->N;
    double U[3] = {0.0, 0.0, 0.0};
    U[d] = sums[9] / Nd;  // mean velocity of the state J is taken on
    // rate groups (e, eps, q, nu, pi, m): d s_g / d s_nu under the set's rules
    double g[6] = {0, 0, 0, 1, 0, 0};
    const double dk8 = dsE_ds(sn, 3.0 / 16.0), dk4 = dsE_ds(sn, 3.0 / 8.0);
    double Lq = NAN, Lm = NAN;
    switch (c->set) {
    case LBM_SET_A: g[0] = g[1] = g[2] = g[4] = g[5] = dk8; break;
    case LBM_SET_B: g[0] = g[1] = g[4] = 1; g[2] = g[5] = dk8; Lq = Lm = 3.0 / 16.0; break;
    case LBM_SET_C: break;
    case LBM_SET_D: g[0] = g[1] = g[4] = 1; g[2] = dk8; g[5] = dk4; Lq = 3.0 / 16.0; Lm = 3.0 / 8.0; break;
    case LBM_SET_E:
        g[0] = g[1] = g[4] = 1;
        g[2] = g[5] = dsE_ds(sn, c->Lambda);
        Lq = Lm = c->Lambda;
        break;
    case LBM_SET_SRT: g[0] = g[1] = g[2] = g[4] = g[5] = 1; break;
    default: break;  // rates given directly: tau acts through s_nu only
    }
    const double dsn_dtau = -1.0 / (tau * tau);
    double dtau = U[d] / (3.0 * Fd);  // explicit: J = nu(tau) U / F
    for (int q = 0; q < 6; ++q) dtau += sums[q] * g[q] * dsn_dtau;
    out->dk_dtau = dtau;
    if (isfinite(Lq)) {
        out->dk_dLambda_q = sums[2] * dsE_dL(sn, Lq);
        out->dk_dLambda_m = sums[5] * dsE_dL(sn, Lm);
        out->dk_dLambda = out->dk_dLambda_q + out->dk_dLambda_m;
    } else {
        out->dk_dLambda = out->dk_dLambda_q = out->dk_dLambda_m = NAN;
    }
    for (int a = 0; a < 3; ++a) out->dk_dF[a] = sums[6 + a];
    // explicit: U_d carries F_d/2 at every fluid node, and J divides by F_d
    out->dk_dF[d] += nu * ((double)c->Nf / (2.0 * Nd)) / Fd - nu * U[d] / (Fd * Fd);
    for (int q = 0; q < 6; ++q) out->dk_ds[q] = sums[q];
    out->k = nu * U[d] / Fd;
    out->iterations = iters;
    out->residual = resid;
}

static int drive_axis(const lbm_ctx *c) {
    int d = 0;
    for (int a = 1; a < 3; ++a)
        if (fabs(c->F[a]) > fabs(c->F[d])) d = a;
    return d;
}

int lbm_adjoint(lbm_ctx *c, double tol, int64_t max_iter, lbm_grad *out) {
    if (!c || !out || !(tol >= 0.0) || max_iter < 1) return LBM_EINVAL;
    if (!c->converged || c->opt.bounceback != 0 || bounded(c)) return LBM_ENOSTATE;
    const int d = drive_axis(c);
    if (c->F[d] == 0.0) return LBM_EINVAL;
    const double nu = (c->tau - 0.5) / 3.0;
    double sums[10];
    int64_t iters = 0;
    double resid = NAN;
    int rc = adjoint_sums(c, tol, max_iter, d, nu / (c->F[d] * (double)c->N), sums, &iters, &resid);
    if (rc) return rc;
    fill_grad(c, d, sums, iters, resid, out);
    return LBM_OK;
}

int lbm_adjoint_transient(lbm_ctx *c, int64_t n, lbm_grad *out) {
    if (!c || !out || n < 1) return LBM_EINVAL;
    if (c->opt.bounceback != 0 || bounded(c)) return LBM_ENOSTATE;
    const int d = drive_axis(c);
    if (c->F[d] == 0.0) return LBM_EINVAL;
    const double nu = (c->tau - 0.5) / 3.0;
    double sums[10];
    c->converged = c->has_conv = false;
    int rc = transient_sums(c, n, d, nu / (c->F[d] * (double)c->N), sums);
    if (rc) return rc;
    fill_grad(c, d, sums, n, NAN, out);
    return LBM_OK;
}

int lbm_mean_velocity(lbm_ctx *c, double U[3]) {
    if (!c || !U) return LBM_EINVAL;
    int nblk = velocity_launch(c, nullptr, true);
    if (nblk > 0)
        launch_finalize(c, nblk, 1.0 / (double)c->N, c->d_U + 3 * 7);
    else
        CK(cudaMemsetAsync(c->d_U + 21, 0, 3 * sizeof(double), c->stream));
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(c->h_U, c->d_U + 21, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (int a = 0; a < 3; ++a) U[a] = c->h_U[a];
    return LBM_OK;
}

int lbm_permeability(lbm_ctx *c, double k[3]) {
    if (!c || !k) return LBM_EINVAL;
    double U[3];
    int rc = lbm_mean_velocity(c, U);
    if (rc) return rc;
    const double nu = (c->tau - 0.5) / 3.0;  // nu = c_s^2 (tau - 1/2)
    for (int a = 0; a < 3; ++a) {
        const double g = drive_of(c, a);
        k[a] = g != 0.0 ? nu * U[a] / g : NAN;
    }
    return LBM_OK;
}

int lbm_velocity(lbm_ctx *c, double *u) {
    if (!c || !u) return LBM_EINVAL;
    double *d_u = nullptr;
    const size_t bytes = sizeof(double) * 3 * (size_t)c->N;
    CK(cudaMalloc(&d_u, bytes));
    cudaError_t e = cudaMemsetAsync(d_u, 0, bytes, c->stream);
    if (e == cudaSuccess) {
        velocity_launch(c, d_u, false);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(u, d_u, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d_u);
    return launch_error(e);
}

int lbm_get_populations(lbm_ctx *c, double *f) {
    if (!c || !f) return LBM_EINVAL;
    double *d_f = nullptr;
    const size_t bytes = sizeof(double) * 19 * (size_t)c->N;
    CK(cudaMalloc(&d_f, bytes));
    launch_export(c, d_f);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(f, d_f, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d_f);
    if (e != cudaSuccess) return launch_error(e);
    std::vector<uint8_t> mask;
    int rc = host_mask(c, mask);
    if (rc != LBM_OK) return rc;
    for (int64_t n = 0; n < c->N; ++n)
        if (mask[(size_t)n])
            for (int i = 0; i < 19; ++i) f[(size_t)i * c->N + n] = weight(i);
    return LBM_OK;
}

int lbm_set_populations(lbm_ctx *c, const double *f) {
    if (!c || !f) return LBM_EINVAL;
    c->converged = c->has_conv = false;
    double *d_f = nullptr;
    const size_t bytes = sizeof(double) * 19 * (size_t)c->N;
    CK(cudaMalloc(&d_f, bytes));
    cudaError_t e = cudaMemcpyAsync(d_f, f, bytes, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) {
        launch_import(c, d_f);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d_f);
    return launch_error(e);
}

int lbm_get_populations_at(lbm_ctx *c, const int64_t *nodes, int64_t count, double *f) {
    if (!c || count < 0 || (count > 0 && (!nodes || !f)) || count > (int64_t(1) << 30))
        return LBM_EINVAL;
    for (int64_t k = 0; k < count; ++k)
        if (nodes[k] < 0 || nodes[k] >= c->N) return LBM_EINVAL;
    if (count == 0) return LBM_OK;
    int64_t *d_nodes = nullptr;
    CK(cudaMalloc(&d_nodes, sizeof(int64_t) * (size_t)count + sizeof(double) * 19 * (size_t)count));
    double *d_f = (double *)(d_nodes + count);
    cudaError_t e = cudaMemcpyAsync(d_nodes, nodes, sizeof(int64_t) * (size_t)count,
                                    cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) {
        launch_export_at(c, d_nodes, (int)count, d_f);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(f, d_f, sizeof(double) * 19 * (size_t)count, cudaMemcpyDeviceToHost,
                            c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d_nodes);
    return launch_error(e);
}

int lbm_link_counts(lbm_ctx *c, int64_t *n_fluid, int64_t links[19]) {
    if (!c) return LBM_EINVAL;
    if (n_fluid) *n_fluid = c->Nf;
    if (links) memcpy(links, c->links, sizeof c->links);
    return LBM_OK;
}

int lbm_sparse_tables(lbm_ctx *c, int32_t *fidx, int32_t *nbr, uint32_t *bb) {
    if (!c) return LBM_EINVAL;
    if (c->opt.layout != LBM_LAYOUT_SPARSE) return LBM_ENOSTATE;
    const size_t Nf = (size_t)c->Nf;
    if (Nf == 0) return LBM_OK;
    if (fidx) CK(cudaMemcpyAsync(fidx, c->d_fidx, 4 * Nf, cudaMemcpyDeviceToHost, c->stream));
    if (nbr) {
        int32_t *d_nbr = nullptr;
        CK(cudaMalloc(&d_nbr, 4 * 18 * Nf));
        int rc = export_sparse_nbr(c, d_nbr);
        cudaError_t e = cudaSuccess;
        if (rc == LBM_OK)
            e = cudaMemcpyAsync(nbr, d_nbr, 4 * 18 * Nf, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        cudaFree(d_nbr);
        if (rc != LBM_OK) return rc;
        if (e != cudaSuccess) return launch_error(e);
    }
    if (bb) CK(cudaMemcpyAsync(bb, c->d_bb, 4 * Nf, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

int64_t lbm_steps_done(const lbm_ctx *c) { return c ? c->steps : -1; }
int64_t lbm_kernel_launches(const lbm_ctx *c) { return c ? c->launches : -1; }

// ------------------------------------------------------------ checkpoints

static const char kMagic[8] = {'L', 'B', 'M', 'G', 'B', '3', '0', '0'};

struct CkptHeader {
    char magic[8];
    int32_t version;
    int32_t dims[3];
    double s[19];
    double F[3];
    int32_t precision, layout, check_interval, linear_eq, fp16_scale_log2, block_size;
    int64_t max_steps;
    int64_t steps;
    int32_t bounceback;
    int32_t stop_rule;
};

// Version 2 appends the bounded-domain settings after the header.
struct CkptDomain {
    int32_t pressure_x, symmetry;
    double rho_in, rho_out;
    int32_t collision, index_width;  // index_width: 0 in files written before it existed
};

int lbm_save(lbm_ctx *c, const char *path) {
    if (!c || !path) return LBM_EINVAL;
    std::vector<uint8_t> mask;
    const int mrc = host_mask(c, mask);
    if (mrc != LBM_OK) return mrc;
    const int64_t units = c->opt.layout == LBM_LAYOUT_SPARSE ? c->Nf : c->N;
    const size_t bytes = c->elem * 19 * (size_t)units;
    std::vector<unsigned char> buf(bytes);
    if (bytes) {
        CK(cudaMemcpyAsync(buf.data(), c->opt.layout == LBM_LAYOUT_AB ? c->d_pop[c->cur] : c->d_pop[0],
                           bytes, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    CkptHeader h;
    memset(&h, 0, sizeof h);
    memcpy(h.magic, kMagic, 8);
    h.version = 2;
    h.dims[0] = c->Lx;
    h.dims[1] = c->Ly;
    h.dims[2] = c->Lz;
    memcpy(h.s, c->s, sizeof h.s);
    memcpy(h.F, c->F, sizeof h.F);
    h.precision = c->opt.precision;
    h.layout = c->opt.layout;
    h.check_interval = c->opt.check_interval;
    h.linear_eq = c->opt.linear_eq;
    h.fp16_scale_log2 = c->opt.fp16_scale_log2;
    h.block_size = c->opt.block_size;
    h.max_steps = c->opt.max_steps;
    h.steps = c->steps;
    h.bounceback = c->opt.bounceback;
    h.stop_rule = c->opt.stop_rule;
    FILE *fp = fopen(path, "wb");
    if (!fp) return LBM_EIO;
    CkptDomain dm{c->opt.pressure_x, c->opt.symmetry, c->opt.rho_in, c->opt.rho_out,
                  c->opt.collision, c->opt.index_width};
    bool ok = fwrite(&h, sizeof h, 1, fp) == 1 && fwrite(&dm, sizeof dm, 1, fp) == 1 &&
              fwrite(mask.data(), 1, (size_t)c->N, fp) == (size_t)c->N &&
              (bytes == 0 || fwrite(buf.data(), 1, bytes, fp) == bytes);
    ok = (fclose(fp) == 0) && ok;
    return ok ? LBM_OK : LBM_EIO;
}

int lbm_load(lbm_ctx **out, const char *path, const lbm_options *opt) {
    if (!out || !path) return LBM_EINVAL;
    *out = nullptr;
    FILE *fp = fopen(path, "rb");
    if (!fp) return LBM_EIO;
    CkptHeader h;
    if (fread(&h, sizeof h, 1, fp) != 1 || memcmp(h.magic, kMagic, 8) != 0 ||
        (h.version != 1 && h.version != 2)) {
        fclose(fp);
        return LBM_EIO;
    }
    CkptDomain dm{0, 0, 1.0, 1.0, 0, 0};  // version 1: periodic, default collision
    if (h.version == 2 && fread(&dm, sizeof dm, 1, fp) != 1) {
        fclose(fp);
        return LBM_EIO;
    }
    const int64_t N = (int64_t)h.dims[0] * h.dims[1] * h.dims[2];
    if (h.dims[0] <= 0 || h.dims[1] <= 0 || h.dims[2] <= 0 || N >= (int64_t(1) << 31)) {
        fclose(fp);
        return LBM_EIO;
    }
    std::vector<uint8_t> mask((size_t)N);
    if (fread(mask.data(), 1, (size_t)N, fp) != (size_t)N) {
        fclose(fp);
        return LBM_EIO;
    }
    lbm_options o;
    lbm_default_options(&o);
    if (opt) o.cuda_stream = opt->cuda_stream;
    o.precision = h.precision;
    o.layout = h.layout;
    o.check_interval = h.check_interval;
    o.linear_eq = h.linear_eq;
    o.fp16_scale_log2 = h.fp16_scale_log2;
    o.block_size = h.block_size;
    o.max_steps = h.max_steps;
    o.stop_rule = h.stop_rule;
    o.bounceback = h.bounceback;
    o.pressure_x = dm.pressure_x;
    o.symmetry = dm.symmetry;
    o.rho_in = dm.rho_in;
    o.rho_out = dm.rho_out;
    o.collision = dm.collision;
    o.index_width = dm.index_width;
    lbm_ctx *c = nullptr;
    int rc = lbm_create_rates(&c, mask.data(), h.dims, h.s, h.F, &o);
    if (rc != LBM_OK) {
        fclose(fp);
        return rc;
    }
    const int64_t units = c->opt.layout == LBM_LAYOUT_SPARSE ? c->Nf : c->N;
    const size_t bytes = c->elem * 19 * (size_t)units;
    std::vector<unsigned char> buf(bytes);
    bool ok = bytes == 0 || fread(buf.data(), 1, bytes, fp) == bytes;
    fclose(fp);
    if (!ok) {
        lbm_destroy(c);
        return LBM_EIO;
    }
    if (bytes) {
        cudaError_t e = cudaMemcpyAsync(c->d_pop[0], buf.data(), bytes, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) {
            lbm_destroy(c);
            return launch_error(e);
        }
    }
    c->cur = 0;
    c->steps = h.steps;
    *out = c;
    return LBM_OK;
}

const char *lbm_strerror(int code) {
    switch (code) {
    case LBM_OK: return "success";
    case LBM_EINVAL: return "invalid argument";
    case LBM_ENOMEM: return "out of memory";
    case LBM_ECUDA: return "CUDA runtime error";
    case LBM_ENOTCONV: return "not converged within max_steps";
    case LBM_EUNSTABLE: return "non-finite density or velocity";
    case LBM_ETIMEOUT: return "bounded device wait expired";
    case LBM_ENOSTATE: return "operation not available in this state or layout";
    case LBM_EIO: return "checkpoint I/O error";
    default: return "unknown error";
    }
}

const char *lbm_last_cuda_error(void) { return g_cuda_err; }

}  // extern "C"

namespace lbm {
// One chunk of the convergence loop for a batch member that runs with the
// single-lattice kernels: `plain` plain steps, then `nmeas` measuring steps
// into slots 0 .. nmeas - 1 of c->d_U, replayed from the context's chunk
// graphs like lbm_run_to_convergence's chunks.  Advances c->steps.
int enqueue_measured_chunk(lbm_ctx *c, int64_t plain, int nmeas) {
    c->converged = c->has_conv = false;
    return enqueue_chunk(c, plain, 0, nmeas);
}
}  // namespace lbm
