// Host-side state of one lattice context (the opaque lbm_ctx of the C ABI):
// device buffers, options, counters and the cached CUDA graphs of the
// convergence loop.  Device code never sees this structure.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "lbm.h"

namespace lbm {
struct RowWord;

// One captured chunk of the convergence loop: `plain` plain steps, then
// `nmeas` measuring steps into slots first .. first + nmeas - 1, starting at
// parity (AA, sparse) or current array (AB) `phase`.
struct ChunkGraph {
    cudaGraphExec_t exec;
    int64_t plain;
    int first, nmeas, phase;
    int64_t dlaunches;  // launches the chunk makes
    int cur_after;      // AB: current array after the chunk
};
constexpr int kChunkGraphs = 4;
}  // namespace lbm

struct lbm_ctx {
    int Lx, Ly, Lz;
    int64_t N, Nf;
    double s[19];
    double tau;  // 1/s_nu
    double F[3];
    lbm_options opt;
    cudaStream_t stream;
    bool own_stream;
    int device;

    uint8_t *d_mask;      // [N]
    uint32_t *d_lw;       // [N] dense link words (AB, AA)
    int32_t *d_fidx;      // [Nf] sparse: node index of each fluid node
    uint32_t *d_bb;       // [Nf] sparse: bounceback bits
    uint2 *d_nb;          // [Nf] sparse: {node index, bounceback bits} interleaved
    lbm::RowWord *d_rw;   // [Ly*Lz][Wr] sparse: row fluid bits + fluid index base
    int32_t *d_rstart;    // [Ly*Lz + 1] sparse: fluid index of each row's first node
    uint2 *d_orec;        // [Nf] sparse, Lx < 2^13: {padded row, bits | x << 19} (OddMap)
    lbm::RowWord *d_rwp;  // [(Ly+2)*(Lz+2)][Wr] padded row words (OddMap)
    int2 *d_rse;          // [(Ly+2)*(Lz+2)] padded row start/end (OddMap)
    int Wr;               // 32-voxel words per row
    void *d_pop[2];       // populations; AB uses both, AA and SPARSE one
    size_t elem;          // bytes per stored population value
    float fp16_scale;     // 2^S (FP16 storage)
    int cur;              // AB: index of the array holding the current state
    int64_t steps;        // time steps taken
    int64_t links[19];

    double *d_partials;   // [max blocks][3]
    int n_partial_blocks;
    double *d_U;          // [8][3]: reduced mean velocities
    int *d_flag;          // non-finite flag
    double *h_U;          // pinned [8*3 + 2]
    int64_t launches;
    int set;              // lbm_set of the rates, -1 when given directly
    double Lambda;        // Set E magic parameter
    bool converged;       // the stopping rule held and the state has not moved since
    bool has_conv;        // U_conv holds the measure of a finished stopping-rule run
    double U_conv[3];     // the mean velocity that run stopped on
    lbm::ChunkGraph graphs[lbm::kChunkGraphs];  // exec == nullptr: unused
    int next_graph;       // round-robin slot for the next capture
    std::vector<lbm_check> history;  // the checks of the last lbm_run_to_convergence
    int odd_npt;          // sparse odd step: fluid nodes per thread (0: not chosen yet)
};
