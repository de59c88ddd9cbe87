// Block grid shared by the SAP preconditioner and the deflation subspace: the
// simulated lattice is tiled by blocks of 4^4 sites, numbered lexicographically
// by block coordinates (bc0 slowest).  One CTA of 128 threads works on one block;
// thread t owns the t-th even and the t-th odd site of the block.
#pragma once

#include "qxd_common.cuh"

namespace qxd {

constexpr int kBlk = 4;           // block extent
constexpr int kBlkThreads = 128;  // half of the 4^4 block sites
constexpr int kBlkSites = 256;

struct SiteRef {
    int l[4];  // local coordinates in the block
    int x[4];  // global coordinates
    int h;     // half index of the site
};

// block coordinates of block b for nb[] blocks per direction
__device__ __forceinline__ void block_coords(int b, const int nb[4], int bc[4]) {
    bc[3] = b % nb[3];
    b /= nb[3];
    bc[2] = b % nb[2];
    b /= nb[2];
    bc[1] = b % nb[1];
    bc[0] = b / nb[1];
}

// the t-th site of parity p in the block with coordinates bc
__device__ __forceinline__ void block_site(const Geo& g, const int bc[4], int p, int t, SiteRef& s) {
    int r = t;
    const int x3h = r & 1;
    r >>= 1;
    s.l[2] = r & 3;
    r >>= 2;
    s.l[1] = r & 3;
    s.l[0] = r >> 2;
    s.l[3] = 2 * x3h + ((p + s.l[0] + s.l[1] + s.l[2]) & 1);
    for (int mu = 0; mu < 4; ++mu) s.x[mu] = kBlk * bc[mu] + s.l[mu];
    s.h = lex_index(g, s.x) >> 1;
}

// thread index of the local site l within its parity
__device__ __forceinline__ int block_thread(const int l[4]) { return (((l[0] * 4 + l[1]) * 4 + l[2]) * 2) + (l[3] >> 1); }

}  // namespace qxd
