// Shared device definitions of libqxd: complex arithmetic, lattice geometry
// with the C* neighbour map, and the internal (structure-of-arrays) layouts of
// spinors, links and site-diagonal terms.
//
// Internal layout.  Every field is split by parity.  A half-lattice field
// lists the sites of one parity by half index h = lex/2 (lex = lexicographic
// index over the simulated lattice, x0 slowest); because N3 is even this is a
// bijection onto [0, V/2) for each parity.  Components are stored as
// structure of arrays: component chunk c of site h lives at base[c*Vh + h], so
// a warp touching 32 consecutive sites reads 32 consecutive 16-byte chunks.
//
//   spinor FP64 : 12 x double2   (complex k = 3*spin + colour)
//   spinor FP32 :  6 x float4    (complex 2c, 2c+1 in chunk c)
//   spinor BF16 :  3 x uint4     (8 bfloat16 = 4 complex per chunk)
//   links  FP64 : per flavour, 36 x double2 = 4 directions x 9 complex entries of
//                 V(x,mu) = U(x,mu) z(x,mu)^qhat (boundary phase folded in)
//   links  FP32 : 12 x float4 = 4 directions x first two rows of U(x,mu) (third
//                 row rebuilt as the conjugate cross product), plus per flavour
//                 2 x float4 = 4 complex phases z(x,mu)^qhat (boundary phase folded in)
//   diag   FP64 : 36 x double2 = two packed Hermitian 6x6 chiral blocks
//   diag   FP32 : 18 x float4
// Packed Hermitian 6x6 block (36 reals): 6 real diagonal entries, then the 15
// upper off-diagonal entries (0,1),(0,2),..,(0,5),(1,2),..,(4,5) as (re, im).
// Block 0 holds spins 0,1 (gamma5 = +1), block 1 spins 2,3 (gamma5 = -1); the
// block-local index is 3*(spin mod 2) + colour.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <string.h>

#include "df64.cuh"

#define QXD_HD __host__ __device__ __forceinline__

#ifdef __CUDA_ARCH__
#define QXD_LDG(p) __ldg(p)
#else
#define QXD_LDG(p) (*(p))
#endif

namespace qxd {

template <typename T>
struct cplx {
    T re, im;
};

template <typename T> QXD_HD cplx<T> mk(T r, T i) { return cplx<T>{r, i}; }
template <typename T> QXD_HD cplx<T> operator+(cplx<T> a, cplx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T> QXD_HD cplx<T> operator-(cplx<T> a, cplx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <typename T> QXD_HD cplx<T> operator-(cplx<T> a) { return {-a.re, -a.im}; }
template <typename T> QXD_HD cplx<T> operator*(cplx<T> a, cplx<T> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename T> QXD_HD cplx<T> operator*(T s, cplx<T> a) { return {s * a.re, s * a.im}; }
template <typename T> QXD_HD cplx<T> conj(cplx<T> a) { return {a.re, -a.im}; }
// conj(a) * b
template <typename T> QXD_HD cplx<T> cmul_conj(cplx<T> a, cplx<T> b) {
    return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
// i * a
template <typename T> QXD_HD cplx<T> times_i(cplx<T> a) { return {-a.im, a.re}; }
// a + i b, a - i b
template <typename T> QXD_HD cplx<T> add_i(cplx<T> a, cplx<T> b) { return {a.re - b.im, a.im + b.re}; }
template <typename T> QXD_HD cplx<T> sub_i(cplx<T> a, cplx<T> b) { return {a.re + b.im, a.im - b.re}; }
// acc += a * b
template <typename T> QXD_HD void cmac(cplx<T>& acc, cplx<T> a, cplx<T> b) {
    acc.re = fma(a.re, b.re, acc.re);
    acc.re = fma(-a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im);
    acc.im = fma(a.im, b.re, acc.im);
}
// acc += conj(a) * b
template <typename T> QXD_HD void cmac_conj(cplx<T>& acc, cplx<T> a, cplx<T> b) {
    acc.re = fma(a.re, b.re, acc.re);
    acc.re = fma(a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im);
    acc.im = fma(-a.im, b.re, acc.im);
}
template <typename T> QXD_HD T norm2(cplx<T> a) { return a.re * a.re + a.im * a.im; }

// --- geometry ---------------------------------------------------------------
struct Geo {
    int N[4];   // simulated (extended) extents
    int L1;     // physical extent in direction 1 (the C* shift)
    int cstar;  // C* in directions 1..cstar
    int Vh;     // V/2
    long long V;
    int open0;  // open time boundary: no hop and no clover leaf across x0 = N0 - 1 <-> 0
};

// coordinates of the site with half index h and parity p
QXD_HD void site_coords(const Geo& g, int p, int h, int x[4]) {
    int n3h = g.N[3] >> 1;
    int x3h = h % n3h;
    int r = h / n3h;
    x[2] = r % g.N[2];
    r /= g.N[2];
    x[1] = r % g.N[1];
    x[0] = r / g.N[1];
    x[3] = 2 * x3h + ((p + x[0] + x[1] + x[2]) & 1);
}

QXD_HD int lex_index(const Geo& g, const int y[4]) {
    return ((y[0] * g.N[1] + y[1]) * g.N[2] + y[2]) * g.N[3] + y[3];
}

// Lexicographic index of x + sign*mu on the simulated torus.  Direction 1 with C*
// is periodic with period 2 L1 (eq. ext-periodic-bc); crossing the boundary of a
// C* direction k = 2, 3 shifts x1 by L1 (eq. ext-shifted-bc); every other
// direction is periodic (its fermion phase lives in the stored link phase).
QXD_HD int neighbour_lex(const Geo& g, const int x[4], int mu, int sign) {
    int y[4] = {x[0], x[1], x[2], x[3]};
    int v = y[mu] + sign;
    bool crossed = false;
    if (v < 0) { v += g.N[mu]; crossed = true; }
    else if (v >= g.N[mu]) { v -= g.N[mu]; crossed = true; }
    y[mu] = v;
    if (crossed && g.cstar >= 1 && mu >= 2 && mu <= g.cstar) {
        int w = y[1] + g.L1;
        y[1] = (w >= g.N[1]) ? w - g.N[1] : w;
    }
    return lex_index(g, y);
}

// --- bfloat16 packing --------------------------------------------------------
QXD_HD uint32_t pack_bf16x2(float a, float b) {
#ifdef __CUDA_ARCH__
    __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&v);
#else
    // round to nearest even on the host (bit manipulation of IEEE binary32)
    auto cvt = [](float f) -> uint32_t {
        uint32_t u;
        memcpy(&u, &f, 4);
        if ((u & 0x7f800000u) == 0x7f800000u) return (u >> 16) | ((u & 0xffff) ? 0x40u : 0u);
        u += 0x7fffu + ((u >> 16) & 1u);
        return u >> 16;
    };
    return cvt(a) | (cvt(b) << 16);
#endif
}
QXD_HD float u32_as_float(uint32_t u) {
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float f;
    memcpy(&f, &u, 4);
    return f;
#endif
}
QXD_HD float bf16_lo(uint32_t v) { return u32_as_float(v << 16); }
QXD_HD float bf16_hi(uint32_t v) { return u32_as_float(v & 0xffff0000u); }

// --- spinor storage ------------------------------------------------------------
// Real type of the arithmetic and chunk type of the storage of each precision.
template <int P> struct Prec;
template <> struct Prec<0> { using real = double; using chunk = double2; static constexpr int nchunk = 12; };
template <> struct Prec<1> { using real = float;  using chunk = float4;  static constexpr int nchunk = 6; };
template <> struct Prec<2> { using real = float;  using chunk = uint4;   static constexpr int nchunk = 3; };
// FP64 data held as double-float pairs, arithmetic in double-float on the FP32 pipe:
// a complex number is one float4 {re.hi, re.lo, im.hi, im.lo}, the chunk of 16
// bytes that the FP64 layout uses for one complex128
template <> struct Prec<3> { using real = dfl;    using chunk = float4;  static constexpr int nchunk = 12; };

template <int P>
QXD_HD void load_spinor(const typename Prec<P>::chunk* __restrict__ base, int stride, int h,
                        cplx<typename Prec<P>::real> s[12]) {
    if constexpr (P == 0) {
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            double2 v = QXD_LDG(base + (size_t)k * stride + h);
            s[k] = {v.x, v.y};
        }
    } else if constexpr (P == 1) {
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            float4 v = QXD_LDG(base + (size_t)c * stride + h);
            s[2 * c] = {v.x, v.y};
            s[2 * c + 1] = {v.z, v.w};
        }
    } else if constexpr (P == 3) {
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            float4 v = QXD_LDG(base + (size_t)k * stride + h);
            s[k] = {dfl(v.x, v.y), dfl(v.z, v.w)};
        }
    } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            uint4 v = QXD_LDG(base + (size_t)c * stride + h);
            s[4 * c + 0] = {bf16_lo(v.x), bf16_hi(v.x)};
            s[4 * c + 1] = {bf16_lo(v.y), bf16_hi(v.y)};
            s[4 * c + 2] = {bf16_lo(v.z), bf16_hi(v.z)};
            s[4 * c + 3] = {bf16_lo(v.w), bf16_hi(v.w)};
        }
    }
}

template <int P>
QXD_HD void store_spinor(typename Prec<P>::chunk* __restrict__ base, int stride, int h,
                         const cplx<typename Prec<P>::real> s[12]) {
    if constexpr (P == 0) {
#pragma unroll
        for (int k = 0; k < 12; ++k) base[(size_t)k * stride + h] = make_double2(s[k].re, s[k].im);
    } else if constexpr (P == 1) {
#pragma unroll
        for (int c = 0; c < 6; ++c)
            base[(size_t)c * stride + h] = make_float4(s[2 * c].re, s[2 * c].im, s[2 * c + 1].re, s[2 * c + 1].im);
    } else if constexpr (P == 3) {
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const dfl re = df_norm(s[k].re), im = df_norm(s[k].im);
            base[(size_t)k * stride + h] = make_float4(re.hi, re.lo, im.hi, im.lo);
        }
    } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            uint4 v;
            v.x = pack_bf16x2(s[4 * c + 0].re, s[4 * c + 0].im);
            v.y = pack_bf16x2(s[4 * c + 1].re, s[4 * c + 1].im);
            v.z = pack_bf16x2(s[4 * c + 2].re, s[4 * c + 2].im);
            v.w = pack_bf16x2(s[4 * c + 3].re, s[4 * c + 3].im);
            base[(size_t)c * stride + h] = v;
        }
    }
}

// --- Hermitian 6x6 blocks ------------------------------------------------------
// index of the packed upper off-diagonal entry (i < j)
QXD_HD constexpr int herm_off(int i, int j) {
    // rows 0..4 hold 5,4,3,2,1 entries
    return (i * (11 - i)) / 2 + (j - i - 1);
}

// out = A in for a packed Hermitian block a[36]
template <typename T>
QXD_HD void herm6_mul(const T a[36], const cplx<T> in[6], cplx<T> out[6]) {
#pragma unroll
    for (int i = 0; i < 6; ++i) out[i] = a[i] * in[i];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
#pragma unroll
        for (int j = i + 1; j < 6; ++j) {
            const int o = 6 + 2 * herm_off(i, j);
            cplx<T> aij = {a[o], a[o + 1]};
            cmac(out[i], aij, in[j]);
            cmac_conj(out[j], aij, in[i]);
        }
    }
}

// load both packed blocks of a site-diagonal term
template <int P>
QXD_HD void load_diag(const void* __restrict__ base, int stride, int h, typename Prec<P>::real a[72]) {
    if constexpr (P == 0) {
        const double2* b = static_cast<const double2*>(base);
#pragma unroll
        for (int k = 0; k < 36; ++k) {
            double2 v = QXD_LDG(b + (size_t)k * stride + h);
            a[2 * k] = v.x;
            a[2 * k + 1] = v.y;
        }
    } else if constexpr (P == 3) {
        const float4* b = static_cast<const float4*>(base);
#pragma unroll
        for (int k = 0; k < 36; ++k) {
            float4 v = QXD_LDG(b + (size_t)k * stride + h);
            a[2 * k] = dfl(v.x, v.y);
            a[2 * k + 1] = dfl(v.z, v.w);
        }
    } else {
        const float4* b = static_cast<const float4*>(base);
#pragma unroll
        for (int k = 0; k < 18; ++k) {
            float4 v = QXD_LDG(b + (size_t)k * stride + h);
            a[4 * k] = v.x;
            a[4 * k + 1] = v.y;
            a[4 * k + 2] = v.z;
            a[4 * k + 3] = v.w;
        }
    }
}

// s <- diag-term s (both chiral blocks)
template <typename T>
QXD_HD void apply_diag(const T a[72], cplx<T> s[12]) {
    cplx<T> o[6];
    herm6_mul(a, s, o);
#pragma unroll
    for (int i = 0; i < 6; ++i) s[i] = o[i];
    herm6_mul(a + 36, s + 6, o);
#pragma unroll
    for (int i = 0; i < 6; ++i) s[6 + i] = o[i];
}

}  // namespace qxd
