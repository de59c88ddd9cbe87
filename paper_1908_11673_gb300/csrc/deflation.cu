// Inexact deflation with SAP (Sec. 4.4, DFL+SAP+GCR; one subspace per flavour
// slot, hence per charge).
//
//   subspace   Ns fields phi_k, started from given random fields; ninv times
//              phi_k <- M_sap phi_k, each time followed by block orthonormalisation
//              (Gram-Schmidt of the restrictions to every 4^4 block, in k order)
//   P, P^+     P c = sum_{B,k} c_{B,k} phi_k|_B,  (P^+ v)_{B,k} = <phi_k|_B, v>
//   A          little Dirac operator P^+ D P: per block B, nine Ns x Ns blocks
//              (B itself and the blocks across its eight faces)
//   M_dfl v  = P A^-1 P^+ v + M_sap (v - D P A^-1 P^+ v), with A^-1 from restarted
//              GCR on the block grid to a relative residual ctol (one cooperative
//              launch, k_dfl_gcr)
//
// Layout.  The basis is Ns full FP32 fields in the internal layout (even half,
// odd half).  Coarse vectors are complex FP32 arrays [Nb][Ns].  A is stored as
// A[B][s][l][k] = <phi_k|_B, D phi_l|_{B_s}> (s = 0 the block itself, 1 + 2 mu the
// block across the +mu face, 2 + 2 mu across the -mu face), so that the lanes that
// form rows k = 0 .. Ns-1 of A x read consecutive entries.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <vector>

#include "blas.h"
#include "block.cuh"
#include "hop.cuh"
#include "ops.h"
#include "qxd_internal.h"

namespace qxd {

namespace {

constexpr int kDflMaxNs = 32;

struct DflGrid {
    int nb[4];
    int Nb;
    int Vh;
};

// CTA-wide sums of n <= kDflMaxNs complex values per thread; thread 0 writes them
__device__ __forceinline__ void cta_sum_cplx(cplx<float>* v, int n, float2* __restrict__ out, float2* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < n; ++k) {
        float re = v[k].re, im = v[k].im;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            re += __shfl_xor_sync(0xffffffffu, re, o);
            im += __shfl_xor_sync(0xffffffffu, im, o);
        }
        if (lane == 0) sh[warp * kDflMaxNs + k] = make_float2(re, im);
    }
    __syncthreads();
    if (threadIdx.x < n) {
        float2 s = make_float2(0.f, 0.f);
        for (int w = 0; w < kBlkThreads / 32; ++w) {
            const float2 t = sh[w * kDflMaxNs + threadIdx.x];
            s.x += t.x;
            s.y += t.y;
        }
        out[threadIdx.x] = s;
    }
    __syncthreads();
}

__device__ __forceinline__ void dot_acc(const cplx<float> a[12], const cplx<float> b[12], cplx<float>& acc) {
#pragma unroll
    for (int i = 0; i < 12; ++i) {
        acc.re += a[i].re * b[i].re + a[i].im * b[i].im;
        acc.im += a[i].re * b[i].im - a[i].im * b[i].re;
    }
}

// out[B][k] = <X_k|_B, v|_B> for k < nk; X_k = X + k * fstride (full FP32 fields)
__global__ void __launch_bounds__(kBlkThreads) k_dfl_dots(Geo g, DflGrid G, const float4* __restrict__ X,
                                                          size_t fstride, int nk, const float4* __restrict__ v,
                                                          float2* __restrict__ out) {
    __shared__ float2 sh[kBlkThreads / 32 * kDflMaxNs];
    int bc[4];
    block_coords(blockIdx.x, G.nb, bc);
    SiteRef se, so;
    block_site(g, bc, 0, threadIdx.x, se);
    block_site(g, bc, 1, threadIdx.x, so);
    const int Vh = g.Vh;
    cplx<float> ve[12], vo[12], x[12];
    load_spinor<1>(v, Vh, se.h, ve);
    load_spinor<1>(v + 6 * (size_t)Vh, Vh, so.h, vo);
    cplx<float> acc[kDflMaxNs];
    for (int k = 0; k < nk; ++k) {
        acc[k] = {0.f, 0.f};
        const float4* Xk = X + (size_t)k * fstride;
        load_spinor<1>(Xk, Vh, se.h, x);
        dot_acc(x, ve, acc[k]);
        load_spinor<1>(Xk + 6 * (size_t)Vh, Vh, so.h, x);
        dot_acc(x, vo, acc[k]);
    }
    cta_sum_cplx(acc, nk, out + (size_t)blockIdx.x * nk, sh);
}

// y = sign * sum_{k < nk} c[B][k] X_k (+ y if accumulate) on every block B
__global__ void __launch_bounds__(kBlkThreads) k_dfl_prolong(Geo g, DflGrid G, const float4* __restrict__ X,
                                                             size_t fstride, int nk, const float2* __restrict__ c,
                                                             float sign, int accumulate, float4* __restrict__ y) {
    __shared__ float2 cs[kDflMaxNs];
    if (threadIdx.x < nk) cs[threadIdx.x] = c[(size_t)blockIdx.x * nk + threadIdx.x];
    __syncthreads();
    int bc[4];
    block_coords(blockIdx.x, G.nb, bc);
    const int Vh = g.Vh;
    for (int p = 0; p < 2; ++p) {
        SiteRef s;
        block_site(g, bc, p, threadIdx.x, s);
        const size_t off = (size_t)p * 6 * Vh;
        cplx<float> acc[12], x[12];
        if (accumulate) load_spinor<1>(y + off, Vh, s.h, acc);
        else
            for (int i = 0; i < 12; ++i) acc[i] = {0.f, 0.f};
        for (int k = 0; k < nk; ++k) {
            load_spinor<1>(X + (size_t)k * fstride + off, Vh, s.h, x);
            const cplx<float> ck = {sign * cs[k].x, sign * cs[k].y};
#pragma unroll
            for (int i = 0; i < 12; ++i) cmac(acc[i], ck, x[i]);
        }
        store_spinor<1>(y + off, Vh, s.h, acc);
    }
}

// x|_B <- x|_B / |x|_B| on every block
__global__ void __launch_bounds__(kBlkThreads) k_dfl_normalise(Geo g, DflGrid G, float4* __restrict__ x) {
    __shared__ float2 sh[kBlkThreads / 32 * kDflMaxNs];
    __shared__ float2 nrm;
    int bc[4];
    block_coords(blockIdx.x, G.nb, bc);
    SiteRef se, so;
    block_site(g, bc, 0, threadIdx.x, se);
    block_site(g, bc, 1, threadIdx.x, so);
    const int Vh = g.Vh;
    cplx<float> e[12], o[12];
    load_spinor<1>(x, Vh, se.h, e);
    load_spinor<1>(x + 6 * (size_t)Vh, Vh, so.h, o);
    cplx<float> acc[1] = {{0.f, 0.f}};
    dot_acc(e, e, acc[0]);
    dot_acc(o, o, acc[0]);
    cta_sum_cplx(acc, 1, &nrm, sh);
    const float f = nrm.x > 0.f ? rsqrtf(nrm.x) : 0.f;
#pragma unroll
    for (int i = 0; i < 12; ++i) {
        e[i] = f * e[i];
        o[i] = f * o[i];
    }
    store_spinor<1>(x, Vh, se.h, e);
    store_spinor<1>(x + 6 * (size_t)Vh, Vh, so.h, o);
}

struct DflOpDev {
    const float4* U32[2];
    const float4* Z32[2];
    const float4* A[2];
};

// -1/2 (1 - gamma_mu) V(x,mu) f(x+mu) (FWD) or -1/2 (1 + gamma_mu) V(x-mu,mu)^+ f(x-mu),
// f an opposite-parity half field, neighbour half index hn; added to acc
template <int MU, bool FWD>
__device__ __forceinline__ void hop_term(const Geo& g, const DflOpDev& d, int p, int h, int hn,
                                         const float4* __restrict__ f, cplx<float> acc[12]) {
    cplx<float> v[12], t[12];
    Half<float> hp, o;
    Mat3<float> m;
    cplx<float> z;
    load_spinor<1>(f, g.Vh, hn, v);
    project<MU, FWD>(v, hp);
    if (FWD) {
        load_link32(d.U32[p], d.Z32[p], g.Vh, MU, h, m, z);
        mul_half<false>(m, hp, o);
    } else {
        load_link32(d.U32[1 - p], d.Z32[1 - p], g.Vh, MU, hn, m, z);
        mul_half<true>(m, hp, o);
    }
#pragma unroll
    for (int sp = 0; sp < 2; ++sp)
#pragma unroll
        for (int c = 0; c < 3; ++c) o.a[sp][c] = FWD ? z * o.a[sp][c] : cmul_conj(z, o.a[sp][c]);
#pragma unroll
    for (int i = 0; i < 12; ++i) t[i] = {0.f, 0.f};
    reconstruct<MU, FWD>(o, t);
#pragma unroll
    for (int i = 0; i < 12; ++i) acc[i] = acc[i] + (-0.5f) * t[i];
}

// the part of (D phi_l)(x) coming from slot s: s = 0 the site term and the hops
// within the block; s = 1 + 2 mu (2 + 2 mu) the hop from x + mu (x - mu) if that
// site lies in another block, else nothing
__device__ __forceinline__ void slot_term(const Geo& g, const DflOpDev& d, const SiteRef& s, int p, int slot,
                                          const float4* __restrict__ phi, cplx<float> acc[12]) {
    const int Vh = g.Vh;
    const float4* fo = phi + (size_t)(1 - p) * 6 * Vh;  // opposite parity half
#pragma unroll
    for (int i = 0; i < 12; ++i) acc[i] = {0.f, 0.f};
    if (slot == 0) {
        cplx<float> v[12];
        load_spinor<1>(phi + (size_t)p * 6 * Vh, Vh, s.h, v);
        float a[72];
        load_diag<1>(d.A[p], Vh, s.h, a);
        apply_diag(a, v);
#pragma unroll
        for (int i = 0; i < 12; ++i) acc[i] = v[i];
#define QXD_INNER(MU)                                                                          \
    if (s.l[MU] + 1 < kBlk) hop_term<MU, true>(g, d, p, s.h, neighbour_lex(g, s.x, MU, +1) >> 1, fo, acc); \
    if (s.l[MU] > 0) hop_term<MU, false>(g, d, p, s.h, neighbour_lex(g, s.x, MU, -1) >> 1, fo, acc);
        QXD_INNER(0) QXD_INNER(1) QXD_INNER(2) QXD_INNER(3)
#undef QXD_INNER
        return;
    }
    const int mu = (slot - 1) >> 1;
    const bool fwd = ((slot - 1) & 1) == 0;
    if (fwd ? s.l[mu] != kBlk - 1 : s.l[mu] != 0) return;
    const int hn = neighbour_lex(g, s.x, mu, fwd ? +1 : -1) >> 1;
    switch (slot) {
        case 1: hop_term<0, true>(g, d, p, s.h, hn, fo, acc); break;
        case 2: hop_term<0, false>(g, d, p, s.h, hn, fo, acc); break;
        case 3: hop_term<1, true>(g, d, p, s.h, hn, fo, acc); break;
        case 4: hop_term<1, false>(g, d, p, s.h, hn, fo, acc); break;
        case 5: hop_term<2, true>(g, d, p, s.h, hn, fo, acc); break;
        case 6: hop_term<2, false>(g, d, p, s.h, hn, fo, acc); break;
        case 7: hop_term<3, true>(g, d, p, s.h, hn, fo, acc); break;
        default: hop_term<3, false>(g, d, p, s.h, hn, fo, acc); break;
    }
}

// A[B][s][l][k] = <phi_k|_B, (slot-s part of D phi_l)|_B> for one l, all blocks and slots
__global__ void __launch_bounds__(kBlkThreads) k_dfl_little(Geo g, DflGrid G, DflOpDev d, const float4* __restrict__ X,
                                                            size_t fstride, int Ns, int l, float2* __restrict__ A) {
    __shared__ float2 sh[kBlkThreads / 32 * kDflMaxNs];
    int bc[4];
    block_coords(blockIdx.x, G.nb, bc);
    SiteRef se, so;
    block_site(g, bc, 0, threadIdx.x, se);
    block_site(g, bc, 1, threadIdx.x, so);
    const int Vh = g.Vh;
    const float4* phi = X + (size_t)l * fstride;
    for (int slot = 0; slot < 9; ++slot) {
        cplx<float> te[12], to[12], x[12];
        slot_term(g, d, se, 0, slot, phi, te);
        slot_term(g, d, so, 1, slot, phi, to);
        cplx<float> acc[kDflMaxNs];
        for (int k = 0; k < Ns; ++k) {
            acc[k] = {0.f, 0.f};
            load_spinor<1>(X + (size_t)k * fstride, Vh, se.h, x);
            dot_acc(x, te, acc[k]);
            load_spinor<1>(X + (size_t)k * fstride + 6 * (size_t)Vh, Vh, so.h, x);
            dot_acc(x, to, acc[k]);
        }
        cta_sum_cplx(acc, Ns, A + (((size_t)blockIdx.x * 9 + slot) * Ns + l) * Ns, sh);
    }
}

// ---- little-system solver: restarted GCR on the block grid in one cooperative launch ----
//
// A x = b (FP32 vectors [Nb][Ns], sums in FP64), x from zero, restarted every nkv steps, until
// |b - A x| <= tol |b| or nmx steps.  Step k of a cycle, with w_j, p_j (j < k) the orthonormal
// directions of the cycle and r orthogonal to every w_j:
//   phase 1  w = A r; partial sums of c_j = <w_j, w>, |w|^2 and <w, r>       (barrier)
//   phase 2  |w'|^2 = |w|^2 - sum_j |c_j|^2 for w' = w - sum_j c_j w_j, and <w', r> = <w, r>;
//            w_k = w' / |w'|, p_k = (r - sum_j c_j p_j) / |w'|, alpha = <w_k, r>,
//            x += alpha p_k, r -= alpha w_k; partial sums of |r|^2            (barrier)
// When |w'|^2 < cancel |w|^2 (cancellation; cancel = 0.01) w' and its products are formed
// explicitly first, with one more barrier.  Every CTA reduces the per-CTA partial sums itself, in the same
// order, so that all CTAs take the same decisions.  The grid barrier polls with a limit; a
// CTA that gives up records the error and leaves, and the others then give up at their next
// barrier.
constexpr int kCgThreads = 512;
constexpr int kCgWarps = kCgThreads / 32;
constexpr int kCgMaxK = 32;                // restart length bound
constexpr int kCgPart = 68;                // doubles per CTA and partial-sum region
constexpr long long kCgSpin = 1ll << 22;   // barrier polls before giving up

struct CgBar {
    unsigned count, gen;
    int err, pad;
};
struct CgStat {
    int iters, err;
    double relres;
};
struct CgArgs {
    DflGrid G;
    int Ns, nkv, nmx;
    double tol2;
    double cancel;  // explicit norm when |w'|^2 < cancel |w|^2
    const int* nbr;
    const float2* A;
    const float2* b;
    float2* x;
    float2* r;
    float2* P;  // [nkv][Nb * Ns]
    float2* W;  // [nkv][Nb * Ns]
    double* part;  // [3][gridDim.x][kCgPart]
    CgBar* bar;
    CgStat* stat;
};

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// grid-wide barrier; false if this CTA gave up waiting or another CTA did before
__device__ bool cg_sync(CgBar* b) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int good = 1;
        const unsigned g = ld_acquire_gpu(&b->gen);
        __threadfence();
        if (atomicAdd(&b->count, 1u) == gridDim.x - 1) {
            atomicExch(&b->count, 0u);
            __threadfence();
            atomicAdd(&b->gen, 1u);
        } else {
            long long polls = 0;
            while (ld_acquire_gpu(&b->gen) == g) {
                if (++polls > kCgSpin) {
                    atomicExch(&b->err, 1);
                    good = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        if (*reinterpret_cast<volatile int*>(&b->err)) good = 0;
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

// FP64 sum of v over the CTA (the same order on every CTA); every thread gets it
__device__ double cg_cta_sum(double v, double* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < kCgWarps; ++w) s += sh[w];
    __syncthreads();
    return s;
}

// out[c] = sum over CTAs i = 0, 1, ... of part[i][c], into shared memory (tmp: kCgThreads
// doubles), for ncol columns: c = 0 .. split - 1 and 64, 65, ... after them (split = ncol:
// the first ncol); the same thread mapping and order on every CTA
__device__ void cg_reduce(const double* part, int ncol, int split, double* out, double* tmp) {
    const int q = min(kCgThreads / ncol, 32);
    const int t = threadIdx.x, cc = t % ncol, grp = t / ncol;
    const int c = cc < split ? cc : 64 + cc - split;
    if (grp < q) {
        double s = 0.0;
#pragma unroll 4
        for (int i = grp; i < (int)gridDim.x; i += q) s += part[(size_t)i * kCgPart + c];
        tmp[grp * ncol + cc] = s;
    }
    __syncthreads();
    if (t < ncol) {
        double s = 0.0;
        for (int g = 0; g < q; ++g) s += tmp[g * ncol + t];
        out[c] = s;
    }
    __syncthreads();
}

// one halving step of the warp transpose-sum: M entries -> M/2, lanes with bit O set keep the
// upper half
template <int M, int O>
__device__ __forceinline__ void halve(float (&v)[2 * kCgMaxK]) {
    const bool up = (threadIdx.x & O) != 0;
#pragma unroll
    for (int i = 0; i < M / 2; ++i) {
        const float send = up ? v[i] : v[i + M / 2];
        const float keep = up ? v[i + M / 2] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, O);
    }
}

// phase 1: w = A r into W[k]; partial sums of <W_j, w> (j < k), |w|^2 and <w, r> -> part.
// A warp takes blocks B = B0, B0 + S, ...: for each, its lanes stage the nine neighbour
// blocks' entries of r in shared memory (xs, 9 Ns per warp), then lane (grp, col) forms row
// col of A r over the rows l = grp (mod ng) of the nine Ns x Ns blocks, three rows (27 loads)
// at a time.  The sums then run over the warp's entries with all 32 lanes.
__device__ void cg_phase1(const CgArgs& a, int k, float* sred, float2* xs) {
    const int Ns = a.Ns;
    const size_t n = (size_t)a.G.Nb * Ns;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ng = 32 / Ns;  // rows of A handled side by side
    const int grp = lane / Ns, col = lane - grp * Ns;
    const float2* r = a.r;
    const int B0 = blockIdx.x * kCgWarps + warp, S = gridDim.x * kCgWarps;
    for (int B = B0; B < a.G.Nb; B += S) {
        for (int i = lane; i < 9 * Ns; i += 32) {
            const int sl = i / Ns;
            xs[i] = r[(size_t)__ldg(a.nbr + (size_t)B * 9 + sl) * Ns + (i - sl * Ns)];
        }
        __syncwarp();
        float ar = 0.f, ai = 0.f;
        if (grp < ng) {
            const float2* AB = a.A + (size_t)B * 9 * Ns * Ns + col;
            for (int l0 = grp; l0 < Ns; l0 += 3 * ng) {
                float2 av[3][9];
#pragma unroll
                for (int u = 0; u < 3; ++u) {
                    const int l = l0 + u * ng;
#pragma unroll
                    for (int sl = 0; sl < 9; ++sl)
                        av[u][sl] = l < Ns ? __ldg(AB + ((size_t)sl * Ns + l) * Ns) : make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int u = 0; u < 3; ++u) {
                    const int l = min(l0 + u * ng, Ns - 1);  // av is zero past the last row
#pragma unroll
                    for (int sl = 0; sl < 9; ++sl) {
                        const float2 xv = xs[sl * Ns + l];
                        ar += av[u][sl].x * xv.x - av[u][sl].y * xv.y;
                        ai += av[u][sl].x * xv.y + av[u][sl].y * xv.x;
                    }
                }
            }
        }
        const float ar0 = ar, ai0 = ai;
        for (int g = 1; g < ng; ++g) {
            ar += __shfl_sync(0xffffffffu, ar0, lane + g * Ns);
            ai += __shfl_sync(0xffffffffu, ai0, lane + g * Ns);
        }
        if (lane < Ns) a.W[(size_t)k * n + (size_t)B * Ns + lane] = make_float2(ar, ai);
        __syncwarp();  // xs reused; W[k] entries read by other lanes below
    }
    float v[2 * kCgMaxK];
#pragma unroll
    for (int j = 0; j < 2 * kCgMaxK; ++j) v[j] = 0.f;
    float ww = 0.f, wrr = 0.f, wri = 0.f;
    const int nbw = B0 < a.G.Nb ? (a.G.Nb - B0 + S - 1) / S : 0;  // blocks of this warp
    for (int f = lane; f < nbw * Ns; f += 32) {
        const int i = f / Ns;
        const size_t e = (size_t)(B0 + i * S) * Ns + (f - i * Ns);
        const float2 w = a.W[(size_t)k * n + e];
        const float2 rv = r[e];
        ww += w.x * w.x + w.y * w.y;
        wrr += w.x * rv.x + w.y * rv.y;  // <w, r> = conj(w) r
        wri += w.x * rv.y - w.y * rv.x;
#pragma unroll
        for (int j = 0; j < kCgMaxK; ++j)
            if (j < k) {
                const float2 wj = a.W[(size_t)j * n + e];
                v[2 * j] += wj.x * w.x + wj.y * w.y;  // <W_j, w>
                v[2 * j + 1] += wj.x * w.y - wj.y * w.x;
            }
    }
    halve<64, 16>(v);
    halve<32, 8>(v);
    halve<16, 4>(v);
    halve<8, 2>(v);
    halve<4, 1>(v);  // lane l now holds the warp totals of <W_l, w> in v[0], v[1]
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ww += __shfl_xor_sync(0xffffffffu, ww, o);
        wrr += __shfl_xor_sync(0xffffffffu, wrr, o);
        wri += __shfl_xor_sync(0xffffffffu, wri, o);
    }
    sred[warp * kCgPart + 2 * lane] = v[0];
    sred[warp * kCgPart + 2 * lane + 1] = v[1];
    if (lane == 0) {
        sred[warp * kCgPart + 64] = ww;
        sred[warp * kCgPart + 65] = wrr;
        sred[warp * kCgPart + 66] = wri;
    }
    __syncthreads();
    if (threadIdx.x < 67) {
        double s = 0.0;
        for (int w = 0; w < kCgWarps; ++w) s += (double)sred[w * kCgPart + threadIdx.x];
        a.part[(size_t)blockIdx.x * kCgPart + threadIdx.x] = s;
    }
}

// phase 2 over every entry e: w = (W_k - sum_{j < nj} c_j W_j) inv, p = (src - sum_{j < nj} c_j P_j) inv;
// with update: W_k = w, P_k = p, x += alpha p, r -= alpha w, and the CTA's |r|^2 into part;
// without: W_k = w, P_k = p, and the CTA's |w|^2 and <w, r> into part
__device__ void cg_phase2(const CgArgs& a, int k, int nj, const float2* cf, float inv, float2 alpha,
                          const float2* src, bool update, double* part, double* shd) {
    const size_t n = (size_t)a.G.Nb * a.Ns;
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
    for (size_t e = (size_t)blockIdx.x * kCgThreads + threadIdx.x; e < n; e += (size_t)gridDim.x * kCgThreads) {
        float2 w = a.W[(size_t)k * n + e];
        float2 p = src[e];
#pragma unroll 4
        for (int j = 0; j < nj; ++j) {
            const float2 c = cf[j], wj = a.W[(size_t)j * n + e], pj = a.P[(size_t)j * n + e];
            w.x -= c.x * wj.x - c.y * wj.y;
            w.y -= c.x * wj.y + c.y * wj.x;
            p.x -= c.x * pj.x - c.y * pj.y;
            p.y -= c.x * pj.y + c.y * pj.x;
        }
        w = make_float2(w.x * inv, w.y * inv);
        p = make_float2(p.x * inv, p.y * inv);
        a.W[(size_t)k * n + e] = w;
        a.P[(size_t)k * n + e] = p;
        float2 rv = a.r[e];
        if (update) {
            float2 xv = a.x[e];
            xv.x += alpha.x * p.x - alpha.y * p.y;
            xv.y += alpha.x * p.y + alpha.y * p.x;
            rv.x -= alpha.x * w.x - alpha.y * w.y;
            rv.y -= alpha.x * w.y + alpha.y * w.x;
            a.x[e] = xv;
            a.r[e] = rv;
            s0 += rv.x * rv.x + rv.y * rv.y;
        } else {
            s0 += w.x * w.x + w.y * w.y;
            s1 += w.x * rv.x + w.y * rv.y;
            s2 += w.x * rv.y - w.y * rv.x;
        }
    }
    const double t0 = cg_cta_sum(s0, shd);
    if (update) {
        if (threadIdx.x == 0) part[(size_t)blockIdx.x * kCgPart] = t0;
        return;
    }
    const double t1 = cg_cta_sum(s1, shd), t2 = cg_cta_sum(s2, shd);
    if (threadIdx.x == 0) {
        part[(size_t)blockIdx.x * kCgPart] = t0;
        part[(size_t)blockIdx.x * kCgPart + 1] = t1;
        part[(size_t)blockIdx.x * kCgPart + 2] = t2;
    }
}

__global__ void __launch_bounds__(kCgThreads, 1) k_dfl_gcr(CgArgs a) {
    __shared__ float sred[kCgWarps * kCgPart];
    __shared__ float2 xs[kCgWarps * 9 * kCgMaxK];
    __shared__ double red[kCgPart], tmp[kCgThreads];
    __shared__ double shd[kCgWarps];
    __shared__ float2 cf[kCgMaxK];
    __shared__ float coef[4];  // inv, alpha.re, alpha.im, mode
    const size_t n = (size_t)a.G.Nb * a.Ns;
    double* part0 = a.part;                                // phase 1 sums
    double* part1 = a.part + (size_t)gridDim.x * kCgPart;  // |r|^2
    double* part2 = part1 + (size_t)gridDim.x * kCgPart;   // explicit |w'|^2, <w', r>
    // x = 0, r = b, |b|^2
    float s = 0.f;
    for (size_t e = (size_t)blockIdx.x * kCgThreads + threadIdx.x; e < n; e += (size_t)gridDim.x * kCgThreads) {
        const float2 bv = a.b[e];
        a.r[e] = bv;
        a.x[e] = make_float2(0.f, 0.f);
        s += bv.x * bv.x + bv.y * bv.y;
    }
    const double bs = cg_cta_sum(s, shd);
    if (threadIdx.x == 0) part1[(size_t)blockIdx.x * kCgPart] = bs;
    int it = 0;
    double bb = 0.0, rr = 0.0;
    bool ok = cg_sync(a.bar);
    if (ok) {
        cg_reduce(part1, 1, 1, red, tmp);
        bb = rr = red[0];
    }
    for (int k = 0; ok && bb > 0.0 && it < a.nmx && rr > a.tol2 * bb; k = (k + 1 == a.nkv) ? 0 : k + 1) {
        cg_phase1(a, k, sred, xs + (threadIdx.x >> 5) * 9 * kCgMaxK);
        if (!(ok = cg_sync(a.bar))) break;
        cg_reduce(part0, 2 * k + 3, 2 * k, red, tmp);
        if (threadIdx.x == 0) {
            const double ww = red[64];
            double cc = 0.0;
            for (int j = 0; j < k; ++j) {
                cc += red[2 * j] * red[2 * j] + red[2 * j + 1] * red[2 * j + 1];
                cf[j] = make_float2((float)red[2 * j], (float)red[2 * j + 1]);
            }
            const double w2 = ww - cc;
            int mode = 0;  // 0: implicit norm, 1: explicit, 2: breakdown
            if (!(ww > 0.0) || !isfinite(ww)) mode = 2;
            else if (!(w2 >= a.cancel * ww)) mode = 1;
            const double inv = mode == 0 ? 1.0 / sqrt(w2) : 1.0;
            coef[0] = (float)inv;
            coef[1] = (float)(red[65] * inv);
            coef[2] = (float)(red[66] * inv);
            coef[3] = (float)mode;
        }
        __syncthreads();
        const int mode = (int)coef[3];
        if (mode == 2) break;
        if (mode == 1) {
            cg_phase2(a, k, k, cf, 1.f, make_float2(0.f, 0.f), a.r, false, part2, shd);
            if (!(ok = cg_sync(a.bar))) break;
            cg_reduce(part2, 3, 3, red, tmp);
            if (!(red[0] > 0.0) || !isfinite(red[0])) break;
            const double inv = 1.0 / sqrt(red[0]);
            cg_phase2(a, k, 0, cf, (float)inv, make_float2((float)(red[1] * inv), (float)(red[2] * inv)),
                      a.P + (size_t)k * n, true, part1, shd);
        } else {
            cg_phase2(a, k, k, cf, coef[0], make_float2(coef[1], coef[2]), a.r, true, part1, shd);
        }
        if (!(ok = cg_sync(a.bar))) break;
        cg_reduce(part1, 1, 1, red, tmp);
        rr = red[0];
        ++it;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.stat->iters = it;
        a.stat->relres = bb > 0.0 ? sqrt(rr / bb) : 0.0;
    }
    if (threadIdx.x == 0 && !ok) atomicExch(&a.stat->err, 1);
}

DflGrid dfl_grid(const Geo& g) {
    DflGrid G;
    G.Nb = 1;
    for (int mu = 0; mu < 4; ++mu) {
        G.nb[mu] = g.N[mu] / kBlk;
        G.Nb *= G.nb[mu];
    }
    G.Vh = g.Vh;
    return G;
}
DflGrid dfl_grid(const qxd_ctx* ctx) { return dfl_grid(ctx->g); }

size_t field_chunks(const qxd_ctx* ctx) { return (size_t)12 * ctx->g.Vh; }  // float4 per full FP32 field

int launch_dots(qxd_ctx* ctx, const float4* X, int nk, const float4* v, float2* out, cudaStream_t st) {
    const DflGrid G = dfl_grid(ctx);
    ProfScope prof(ctx, "dfl_dots", (double)ctx->g.V * 96 * (nk + 1), st);
    k_dfl_dots<<<G.Nb, kBlkThreads, 0, st>>>(ctx->g, G, X, field_chunks(ctx), nk, v, out);
    QXD_CUDA(ctx, cudaGetLastError());
    return QXD_OK;
}

int launch_prolong(qxd_ctx* ctx, const float4* X, int nk, const float2* c, float sign, int accumulate, float4* y,
                   cudaStream_t st) {
    const DflGrid G = dfl_grid(ctx);
    ProfScope prof(ctx, "dfl_prolong", (double)ctx->g.V * 96 * (nk + 1 + accumulate), st);
    k_dfl_prolong<<<G.Nb, kBlkThreads, 0, st>>>(ctx->g, G, X, field_chunks(ctx), nk, c, sign, accumulate, y);
    QXD_CUDA(ctx, cudaGetLastError());
    return QXD_OK;
}

// block Gram-Schmidt of the basis (classical, twice per vector, then normalised)
int orthonormalise(qxd_ctx* ctx, QxdFlavour& F, cudaStream_t st) {
    const DflGrid G = dfl_grid(ctx);
    void* c;
    QXD_TRY(qxd_ws(ctx, WS_DFL + 0, sizeof(float2) * (size_t)G.Nb * kDflMaxNs, &c));
    const size_t fs = field_chunks(ctx);
    for (int k = 0; k < F.dfl_Ns; ++k) {
        float4* xk = F.dfl_basis + (size_t)k * fs;
        for (int pass = 0; pass < 2 && k > 0; ++pass) {
            QXD_TRY(launch_dots(ctx, F.dfl_basis, k, xk, static_cast<float2*>(c), st));
            QXD_TRY(launch_prolong(ctx, F.dfl_basis, k, static_cast<const float2*>(c), -1.f, 1, xk, st));
        }
        ProfScope prof(ctx, "dfl_normalise", (double)ctx->g.V * 192, st);
        k_dfl_normalise<<<G.Nb, kBlkThreads, 0, st>>>(ctx->g, G, xk);
        QXD_CUDA(ctx, cudaGetLastError());
    }
    return QXD_OK;
}

// block neighbour table [Nb][9] from the lattice neighbour map (C* shifts included)
void neighbour_table(const Geo& g, std::vector<int>& nbr) {
    const DflGrid G = dfl_grid(g);
    nbr.assign((size_t)G.Nb * 9, 0);
    auto block_of = [&](int lex) {
        int x[4];
        int r = lex;
        for (int mu = 3; mu >= 0; --mu) {
            x[mu] = r % g.N[mu];
            r /= g.N[mu];
        }
        int b = 0;
        for (int mu = 0; mu < 4; ++mu) b = b * G.nb[mu] + x[mu] / kBlk;
        return b;
    };
    for (int B = 0; B < G.Nb; ++B) {
        int bc[4], b = B;
        for (int mu = 3; mu >= 0; --mu) {
            bc[mu] = b % G.nb[mu];
            b /= G.nb[mu];
        }
        nbr[(size_t)B * 9] = B;
        for (int mu = 0; mu < 4; ++mu) {
            int x[4];
            for (int nu = 0; nu < 4; ++nu) x[nu] = kBlk * bc[nu];
            x[mu] = kBlk * bc[mu] + kBlk - 1;  // a site on the +mu face
            nbr[(size_t)B * 9 + 1 + 2 * mu] = block_of(neighbour_lex(g, x, mu, +1));
            x[mu] = kBlk * bc[mu];  // a site on the -mu face
            nbr[(size_t)B * 9 + 2 + 2 * mu] = block_of(neighbour_lex(g, x, mu, -1));
        }
    }
}

int assemble_little(qxd_ctx* ctx, int fl, QxdFlavour& F, cudaStream_t st) {
    const DflGrid G = dfl_grid(ctx);
    const Geo& g = ctx->g;
    DflOpDev d;
    for (int p = 0; p < 2; ++p) {
        d.U32[p] = ctx->U32 + (size_t)p * 12 * g.Vh;
        d.Z32[p] = F.Z32 + (size_t)p * 2 * g.Vh;
        d.A[p] = F.C32[0] + (size_t)p * 18 * g.Vh;
    }
    (void)fl;
    for (int l = 0; l < F.dfl_Ns; ++l) {
        ProfScope prof(ctx, "dfl_little", (double)g.V * (96.0 * (9 * F.dfl_Ns + 3) + 224 + 288), st);
        k_dfl_little<<<G.Nb, kBlkThreads, 0, st>>>(g, G, d, F.dfl_basis, field_chunks(ctx), F.dfl_Ns, l, F.dfl_A);
        QXD_CUDA(ctx, cudaGetLastError());
    }
    return QXD_OK;
}

// A^-1 b to a relative residual ctol (restarted GCR, one cooperative launch); the step
// count, residual and barrier status go to F.dfl_stat
int coarse_gcr(qxd_ctx* ctx, const QxdFlavour& F, const float2* b, float2* x, cudaStream_t st) {
    const DflGrid G = dfl_grid(ctx);
    const size_t n = (size_t)G.Nb * F.dfl_Ns;
    const int nkv = F.dfl_cnkv;
    int nsm = 0, per = 0;
    QXD_CUDA(ctx, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device));
    QXD_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_dfl_gcr, kCgThreads, 0));
    if (per < 1 || nsm < 1) return qxd_fail(ctx, QXD_ECUDA, "little-system solver: kernel does not fit on an SM");
    // every CTA resident at once (the grid barrier needs it); QXD_DFL_CTAS caps the count
    // (a test forces several blocks per warp with it)
    int nblk = std::min(per * nsm, (G.Nb + kCgWarps - 1) / kCgWarps);
    if (const char* env = std::getenv("QXD_DFL_CTAS")) {
        const int cap = std::atoi(env);
        if (cap >= 1) nblk = std::min(nblk, cap);
    }
    nblk = std::max(nblk, 1);
    const size_t vb = sizeof(float2) * n;
    const size_t pb = sizeof(double) * 3 * (size_t)nblk * kCgPart;
    void* slab;
    QXD_TRY(qxd_ws(ctx, WS_DFL + 1, pb + vb * (2 * nkv + 1) + sizeof(CgBar), &slab));
    char* base = static_cast<char*>(slab);
    CgArgs a;
    a.G = G;
    a.Ns = F.dfl_Ns;
    a.nkv = nkv;
    a.nmx = F.dfl_cnmx;
    a.tol2 = F.dfl_ctol * F.dfl_ctol;
    a.cancel = 0.01;
    if (const char* env = std::getenv("QXD_DFL_CANCEL")) a.cancel = std::atof(env);  // > 1: always explicit
    a.nbr = F.dfl_nbr;
    a.A = F.dfl_A;
    a.b = b;
    a.x = x;
    a.part = reinterpret_cast<double*>(base);
    a.r = reinterpret_cast<float2*>(base + pb);
    a.P = reinterpret_cast<float2*>(base + pb + vb);
    a.W = reinterpret_cast<float2*>(base + pb + vb * (1 + nkv));
    a.bar = reinterpret_cast<CgBar*>(base + pb + vb * (1 + 2 * nkv));
    a.stat = static_cast<CgStat*>(F.dfl_stat);
    QXD_CUDA(ctx, cudaMemsetAsync(a.bar, 0, sizeof(CgBar), st));
    void* args[] = {&a};
    ProfScope prof(ctx, "dfl_gcr", 0.0, st);
    QXD_CUDA(ctx, cudaLaunchCooperativeKernel((const void*)k_dfl_gcr, dim3(nblk), dim3(kCgThreads), args, 0, st));
    return QXD_OK;
}

}  // namespace

// the last little-system solve's step count and residual (synchronises the stream); an
// error if a grid barrier of any solve since the set-up gave up waiting
int dfl_status(qxd_ctx* ctx, int fl, int* iters, double* relres, cudaStream_t st) {
    const QxdFlavour& F = ctx->fl[fl];
    if (!F.dfl_stat) return QXD_OK;
    CgStat h{};
    QXD_CUDA(ctx, cudaMemcpyAsync(&h, F.dfl_stat, sizeof(CgStat), cudaMemcpyDeviceToHost, st));
    QXD_CUDA(ctx, cudaStreamSynchronize(st));
    if (h.err) return qxd_fail(ctx, QXD_ECUDA, "little-system solver: a grid barrier gave up waiting");
    if (iters) *iters = h.iters;
    if (relres) *relres = h.relres;
    return QXD_OK;
}

// out = M_dfl v on full FP32 fields (v, out distinct)
int dfl_apply_full(qxd_ctx* ctx, int fl, const float4* v, float4* out, int* citers, double* crel, cudaStream_t st) {
    QxdFlavour& F = ctx->fl[fl];
    if (!F.dfl_basis) return qxd_fail(ctx, QXD_ESTATE, "deflation subspace not set up (qxd_dfl_setup)");
    const DflGrid G = dfl_grid(ctx);
    const size_t hb = half_bytes(ctx, QXD_FP32);
    const size_t cvb = sizeof(float2) * (size_t)G.Nb * F.dfl_Ns;
    void *c, *y, *u, *t;
    QXD_TRY(qxd_ws(ctx, WS_DFL + 2, cvb, &c));
    QXD_TRY(qxd_ws(ctx, WS_DFL + 3, cvb, &y));
    QXD_TRY(qxd_ws(ctx, WS_DFL + 4, 2 * hb, &u));
    QXD_TRY(qxd_ws(ctx, WS_DFL + 5, 2 * hb, &t));
    // u = P A^-1 P^+ v
    QXD_TRY(launch_dots(ctx, F.dfl_basis, F.dfl_Ns, v, static_cast<float2*>(c), st));
    QXD_TRY(coarse_gcr(ctx, F, static_cast<const float2*>(c), static_cast<float2*>(y), st));
    if (citers || crel) {
        int it = 0;
        double rel = 0.0;
        QXD_TRY(dfl_status(ctx, fl, &it, &rel, st));
        if (citers) *citers = it;
        if (crel) *crel = rel;
    }
    float4* uf = static_cast<float4*>(u);
    float4* tf = static_cast<float4*>(t);
    QXD_TRY(launch_prolong(ctx, F.dfl_basis, F.dfl_Ns, static_cast<const float2*>(y), 1.f, 0, uf, st));
    // t = v - D u;  out = M_sap t + u
    char* uc = static_cast<char*>(u);
    char* tc = static_cast<char*>(t);
    QXD_TRY(op_Dw(ctx, fl, QXD_FP32, Full{uc, uc + hb}, Full{tc, tc + hb}, st));
    const size_t n2 = 24ull * ctx->g.Vh;
    QXD_TRY(blas_axpby(ctx, 1, 1, n2, 1.0, 0.0, v, -1.0, 0.0, tf, st));
    QXD_TRY(sap_apply_full(ctx, fl, tf, out, st));
    QXD_TRY(blas_axpby(ctx, 1, 1, n2, 1.0, 0.0, uf, 1.0, 0.0, out, st));
    return QXD_OK;
}

// z_e = (M_dfl (r_e, 0))_e on FP32 even fields
int dfl_apply_even(qxd_ctx* ctx, int fl, const void* r_e, void* z_e, cudaStream_t st) {
    const size_t hb = half_bytes(ctx, QXD_FP32);
    void *eta, *psi;
    QXD_TRY(qxd_ws(ctx, WS_DFL + 6, 2 * hb, &eta));
    QXD_TRY(qxd_ws(ctx, WS_DFL + 7, 2 * hb, &psi));
    QXD_CUDA(ctx, cudaMemcpyAsync(eta, r_e, hb, cudaMemcpyDeviceToDevice, st));
    QXD_CUDA(ctx, cudaMemsetAsync(static_cast<char*>(eta) + hb, 0, hb, st));
    QXD_TRY(dfl_apply_full(ctx, fl, static_cast<const float4*>(eta), static_cast<float4*>(psi), nullptr, nullptr, st));
    QXD_CUDA(ctx, cudaMemcpyAsync(z_e, psi, hb, cudaMemcpyDeviceToDevice, st));
    return QXD_OK;
}

void dfl_free(QxdFlavour& F) {
    cudaFree(F.dfl_basis);
    cudaFree(F.dfl_A);
    cudaFree(F.dfl_nbr);
    cudaFree(F.dfl_stat);
    F.dfl_basis = nullptr;
    F.dfl_A = nullptr;
    F.dfl_nbr = nullptr;
    F.dfl_stat = nullptr;
    F.dfl_Ns = 0;
}

}  // namespace qxd

using namespace qxd;

extern "C" {

int qxd_dfl_setup(qxd_ctx* ctx, int fl, const qxd_dfl_params* prm, const void* seeds, void* stream) {
    QXD_TRY(check_fl(ctx, fl));
    if (!prm || !seeds) return qxd_fail(ctx, QXD_EARG, "dfl_setup: NULL argument");
    if (prm->Ns < 1 || prm->Ns > kDflMaxNs) return qxd_fail(ctx, QXD_EARG, "dfl_setup: Ns must be 1..32");
    if (prm->ninv < 0 || prm->ninv > 64) return qxd_fail(ctx, QXD_EARG, "dfl_setup: ninv must be 0..64");
    if (!(prm->ctol > 0.0) || prm->cnmx < 1 || prm->cnkv < 1 || prm->cnkv > 32)
        return qxd_fail(ctx, QXD_EARG, "dfl_setup: need ctol > 0, cnmx >= 1, cnkv in 1..32");
    QXD_TRY(sap_check(ctx));
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    QxdFlavour& F = ctx->fl[fl];
    dfl_free(F);
    const DflGrid G = dfl_grid(ctx);
    const size_t fs = field_chunks(ctx);
    const int Ns = prm->Ns;
    QXD_CUDA(ctx, cudaMalloc(&F.dfl_basis, sizeof(float4) * fs * Ns));
    QXD_CUDA(ctx, cudaMalloc(&F.dfl_A, sizeof(float2) * (size_t)G.Nb * 9 * Ns * Ns));
    QXD_CUDA(ctx, cudaMalloc(&F.dfl_nbr, sizeof(int) * (size_t)G.Nb * 9));
    QXD_CUDA(ctx, cudaMalloc(&F.dfl_stat, sizeof(CgStat)));
    QXD_CUDA(ctx, cudaMemsetAsync(F.dfl_stat, 0, sizeof(CgStat), st));
    F.dfl_Ns = Ns;
    F.dfl_ctol = prm->ctol;
    F.dfl_cnmx = prm->cnmx;
    F.dfl_cnkv = prm->cnkv;
    std::vector<int> nbr;
    neighbour_table(ctx->g, nbr);
    QXD_CUDA(ctx, cudaMemcpyAsync(F.dfl_nbr, nbr.data(), sizeof(int) * nbr.size(), cudaMemcpyHostToDevice, st));
    // seeds: complex64 [Ns][V][4][3] -> internal FP32 fields
    const size_t cb = (size_t)ctx->g.V * 12 * 8;
    const size_t hb = half_bytes(ctx, QXD_FP32);
    const void* din;
    int rc = stage_in(ctx, WS_STAGE_IN, seeds, cb * Ns, &din, st);
    if (rc == QXD_OK) {
        for (int k = 0; k < Ns && rc == QXD_OK; ++k) {
            const char* src = static_cast<const char*>(din) + cb * k;
            char* dst = reinterpret_cast<char*>(F.dfl_basis + fs * k);
            rc = launch_pack(ctx, 1, src, 1, 0, QXD_FP32, dst, 1, st);
            if (rc == QXD_OK) rc = launch_pack(ctx, 1, src, 1, 1, QXD_FP32, dst + hb, 1, st);
        }
    }
    if (rc == QXD_OK) rc = orthonormalise(ctx, F, st);
    void* tmp = nullptr;
    if (rc == QXD_OK) rc = qxd_ws(ctx, WS_DFL + 8, 2 * hb, &tmp);
    for (int i = 0; i < prm->ninv && rc == QXD_OK; ++i) {
        for (int k = 0; k < Ns && rc == QXD_OK; ++k) {
            float4* xk = F.dfl_basis + fs * k;
            rc = sap_apply_full(ctx, fl, xk, static_cast<float4*>(tmp), st);
            if (rc == QXD_OK) {
                cudaError_t e = cudaMemcpyAsync(xk, tmp, 2 * hb, cudaMemcpyDeviceToDevice, st);
                if (e != cudaSuccess) rc = qxd_fail(ctx, QXD_ECUDA, cudaGetErrorString(e));
            }
        }
        if (rc == QXD_OK) rc = orthonormalise(ctx, F, st);
    }
    if (rc == QXD_OK) rc = assemble_little(ctx, fl, F, st);
    if (rc == QXD_OK) {
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = qxd_fail(ctx, QXD_ECUDA, cudaGetErrorString(e));
    }
    if (rc != QXD_OK) dfl_free(F);
    return rc;
}

int qxd_dfl_basis(qxd_ctx* ctx, int fl, int k, void* out, void* stream) {
    QXD_TRY(check_fl(ctx, fl));
    QxdFlavour& F = ctx->fl[fl];
    if (!F.dfl_basis) return qxd_fail(ctx, QXD_ESTATE, "deflation subspace not set up (qxd_dfl_setup)");
    if (k < 0 || k >= F.dfl_Ns || !out) return qxd_fail(ctx, QXD_EARG, "dfl_basis: k out of range or NULL output");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t cb = (size_t)ctx->g.V * 12 * 8;
    const size_t hb = half_bytes(ctx, QXD_FP32);
    void* dout;
    bool host_out;
    QXD_TRY(stage_out(ctx, WS_STAGE_OUT, out, cb, &dout, &host_out));
    const char* src = reinterpret_cast<const char*>(F.dfl_basis + field_chunks(ctx) * k);
    QXD_TRY(launch_unpack(ctx, QXD_FP32, src, 0, 1, dout, 1, 1, st));
    QXD_TRY(launch_unpack(ctx, QXD_FP32, src + hb, 1, 1, dout, 1, 1, st));
    QXD_TRY(finish_out(ctx, out, dout, cb, host_out, st));
    QXD_CUDA(ctx, cudaStreamSynchronize(st));
    return QXD_OK;
}

int qxd_dfl_little(qxd_ctx* ctx, int fl, void* A_out, int* nbr_out, int* nblocks, void* stream) {
    QXD_TRY(check_fl(ctx, fl));
    QxdFlavour& F = ctx->fl[fl];
    if (!F.dfl_basis) return qxd_fail(ctx, QXD_ESTATE, "deflation subspace not set up (qxd_dfl_setup)");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const DflGrid G = dfl_grid(ctx);
    if (nblocks) *nblocks = G.Nb;
    if (A_out)
        QXD_CUDA(ctx, cudaMemcpyAsync(A_out, F.dfl_A, sizeof(float2) * (size_t)G.Nb * 9 * F.dfl_Ns * F.dfl_Ns,
                                      cudaMemcpyDefault, st));
    if (nbr_out)
        QXD_CUDA(ctx, cudaMemcpyAsync(nbr_out, F.dfl_nbr, sizeof(int) * (size_t)G.Nb * 9, cudaMemcpyDefault, st));
    QXD_CUDA(ctx, cudaStreamSynchronize(st));
    return QXD_OK;
}

int qxd_dfl_apply(qxd_ctx* ctx, int fl, const void* in, void* out, qxd_info* info, void* stream) {
    QXD_TRY(check_fl(ctx, fl));
    if (!in || !out) return qxd_fail(ctx, QXD_EARG, "dfl_apply: NULL argument");
    if (!ctx->fl[fl].dfl_basis) return qxd_fail(ctx, QXD_ESTATE, "deflation subspace not set up (qxd_dfl_setup)");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t cb = (size_t)ctx->g.V * 12 * 8;
    const size_t hb = half_bytes(ctx, QXD_FP32);
    void *cin, *cout, *fin, *fout;
    QXD_TRY(qxd_ws(ctx, WS_DFL + 9, cb, &cin));
    QXD_TRY(qxd_ws(ctx, WS_DFL + 10, cb, &cout));
    QXD_TRY(qxd_ws(ctx, WS_DFL + 11, 2 * hb, &fin));
    QXD_TRY(qxd_ws(ctx, WS_DFL + 12, 2 * hb, &fout));
    QXD_CUDA(ctx, cudaMemcpyAsync(cin, in, cb, cudaMemcpyDefault, st));
    char* fi = static_cast<char*>(fin);
    char* fo = static_cast<char*>(fout);
    QXD_TRY(launch_pack(ctx, 1, cin, 1, 0, QXD_FP32, fi, 1, st));
    QXD_TRY(launch_pack(ctx, 1, cin, 1, 1, QXD_FP32, fi + hb, 1, st));
    int it = 0;
    double rel = 0.0;
    QXD_TRY(dfl_apply_full(ctx, fl, reinterpret_cast<const float4*>(fi), reinterpret_cast<float4*>(fo), &it, &rel, st));
    QXD_TRY(launch_unpack(ctx, QXD_FP32, fo, 0, 1, cout, 1, 1, st));
    QXD_TRY(launch_unpack(ctx, QXD_FP32, fo + hb, 1, 1, cout, 1, 1, st));
    QXD_CUDA(ctx, cudaMemcpyAsync(out, cout, cb, cudaMemcpyDefault, st));
    QXD_CUDA(ctx, cudaStreamSynchronize(st));
    if (info) {
        *info = qxd_info{};
        info->iters = it;
        info->true_relres = rel;
    }
    return QXD_OK;
}

int qxd_block_neighbours(const qxd_geom* geom, int* nbr_out, int* nblocks) {
    if (!geom) return QXD_EARG;
    Geo g;
    if (!make_geo(geom, &g)) return QXD_EARG;
    for (int mu = 0; mu < 4; ++mu)
        if (g.N[mu] % (2 * kBlk)) return QXD_EARG;
    const DflGrid G = dfl_grid(g);
    if (nblocks) *nblocks = G.Nb;
    if (nbr_out) {
        std::vector<int> nbr;
        neighbour_table(g, nbr);
        std::copy(nbr.begin(), nbr.end(), nbr_out);
    }
    return QXD_OK;
}

}  // extern "C"
