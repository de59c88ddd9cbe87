// Deterministic grid reductions shared by the vector kernels (blas.cu) and the
// hopping kernel with fused inner products (hop_dots.cu).  Every block writes its
// FP64 partial sums; the last block to finish (a ticket counter) adds all partials
// in block order, so the result is the same on every run for a given grid.
#pragma once

#include <map>
#include <mutex>

#include "blas.h"
#include "qxd_internal.h"

namespace qxd {

constexpr int kRedThreads = 256;

// Grid of a grid-stride kernel: at most one full wave of resident blocks (the
// occupancy of this kernel on this device, looked up once), and no more blocks
// than the work needs.  A fixed grid for a given device and size keeps the
// order of the reduction, and so its result, the same on every run.
template <typename K>
static int wave_blocks(qxd_ctx* ctx, K kernel, int threads, size_t work_per_block, size_t nch) {
    static std::map<const void*, int> per_sm;  // per kernel instantiation
    static std::mutex mu;
    int b_sm;
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = per_sm.find((const void*)kernel);
        if (it == per_sm.end()) {
            int n = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, 0) != cudaSuccess || n < 1) {
                cudaGetLastError();
                n = 1;
            }
            it = per_sm.emplace((const void*)kernel, n).first;
        }
        b_sm = it->second;
    }
    size_t cap = (size_t)b_sm * ctx->nsm;
    if (cap > (size_t)kMaxRedBlocks) cap = kMaxRedBlocks;
    size_t need = (nch + work_per_block - 1) / work_per_block;
    return (int)(need < cap ? (need > 0 ? need : 1) : cap);
}

struct RedOut {
    double* partials;
    unsigned* ticket;
    double* result;
};

static RedOut red_out(qxd_ctx* ctx, int slot) { return RedOut{ctx->red_partials, ctx->red_ticket, ctx->red_result + slot}; }

template <int NC>
__device__ void block_reduce_finish(double v[NC], const RedOut& o) {
    __shared__ double sh[NC][kRedThreads / 32];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        double x = v[c];
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) x += __shfl_down_sync(0xffffffffu, x, s);
        if (lane == 0) sh[c][warp] = x;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            double x = lane < kRedThreads / 32 ? sh[c][lane] : 0.0;
#pragma unroll
            for (int s = 16; s > 0; s >>= 1) x += __shfl_down_sync(0xffffffffu, x, s);
            if (lane == 0) o.partials[(size_t)c * gridDim.x + blockIdx.x] = x;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(o.ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    const int nb = gridDim.x;
    for (int c = 0; c < NC; ++c) {
        double x = 0.0;
        for (int b = threadIdx.x; b < nb; b += blockDim.x) x += __ldcg(o.partials + (size_t)c * nb + b);
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) x += __shfl_down_sync(0xffffffffu, x, s);
        __syncthreads();
        if (lane == 0) sh[0][warp] = x;
        __syncthreads();
        if (warp == 0) {
            x = lane < kRedThreads / 32 ? sh[0][lane] : 0.0;
#pragma unroll
            for (int s = 16; s > 0; s >>= 1) x += __shfl_down_sync(0xffffffffu, x, s);
            if (lane == 0) o.result[c] = x;
        }
    }
    if (threadIdx.x == 0) *o.ticket = 0u;
}

}  // namespace qxd
