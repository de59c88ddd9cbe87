// Double-float ("df64") arithmetic: a real number held as the unevaluated sum
// hi + lo of two floats with |lo| <= ulp(hi) / 2, about 48 significant bits.
// Sums use Knuth's error-free two-sum, products the exact product that one fused
// multiply-add gives (the error of a*b is fma(a, b, -a*b) exactly), each followed
// by a renormalisation; these are the published error-free transformations.
// On GB300 the FP64 pipe runs at 1/64 of the FP32 rate, so an FP64-data stencil
// evaluated in double-float on the FP32 pipe is bound by memory rather than by
// the FP64 units.
//
// Every step goes through the __f*_rn intrinsics, which the compiler never
// contracts into fused multiply-adds or reassociates: the transformations are
// exact only with the rounding of each individual operation.
#pragma once

#include <cuda_runtime.h>

#include <cmath>

#define QXD_DF_HD __host__ __device__ __forceinline__

namespace qxd {

#ifdef __CUDA_ARCH__
#define QXD_FADD(a, b) __fadd_rn(a, b)
#define QXD_FSUB(a, b) __fsub_rn(a, b)
#define QXD_FMUL(a, b) __fmul_rn(a, b)
#define QXD_FFMA(a, b, c) __fmaf_rn(a, b, c)
#else
#define QXD_FADD(a, b) ((a) + (b))
#define QXD_FSUB(a, b) ((a) - (b))
#define QXD_FMUL(a, b) ((a) * (b))
#define QXD_FFMA(a, b, c) fmaf(a, b, c)
#endif

struct dfl {
    float hi, lo;
    dfl() = default;
    QXD_DF_HD constexpr dfl(float h, float l) : hi(h), lo(l) {}
    // nearest double-float of a double (used for constants and for conversions)
    QXD_DF_HD dfl(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
    QXD_DF_HD dfl(int i) : dfl((double)i) {}
};

// s + e = a + b exactly (any magnitudes)
QXD_DF_HD dfl df_two_sum(float a, float b) {
    const float s = QXD_FADD(a, b);
    const float bb = QXD_FSUB(s, a);
    const float e = QXD_FADD(QXD_FSUB(a, QXD_FSUB(s, bb)), QXD_FSUB(b, bb));
    return dfl(s, e);
}
// s + e = a + b exactly, for |a| >= |b|
QXD_DF_HD dfl df_fast_two_sum(float a, float b) {
    const float s = QXD_FADD(a, b);
    const float e = QXD_FSUB(b, QXD_FSUB(s, a));
    return dfl(s, e);
}

// Sums and products are lazy: the error term of the leading parts is kept exactly
// (two-sum, exact product), the trailing parts are added in single precision,
// and the pair is not renormalised, so |lo| may grow to a few ulp(hi) along a
// chain of additions.  df_norm restores |lo| <= ulp(hi) / 2 (before a store).
// Products drop lo * lo; as long as one factor of every product is a freshly
// loaded (normalised) value, as in the stencil, the result holds about 2^-46
// relative accuracy after the ~10^2 operations of one output component.
QXD_DF_HD dfl operator+(dfl a, dfl b) {
    const dfl s = df_two_sum(a.hi, b.hi);
    return dfl(s.hi, QXD_FADD(QXD_FADD(a.lo, b.lo), s.lo));
}
QXD_DF_HD dfl operator-(dfl a) { return dfl(-a.hi, -a.lo); }
QXD_DF_HD dfl operator-(dfl a, dfl b) { return a + (-b); }
QXD_DF_HD dfl operator*(dfl a, dfl b) {
    const float p = QXD_FMUL(a.hi, b.hi);
    float e = QXD_FFMA(a.hi, b.hi, -p);
    e = QXD_FFMA(a.hi, b.lo, e);
    e = QXD_FFMA(a.lo, b.hi, e);
    return dfl(p, e);
}
QXD_DF_HD dfl df_norm(dfl a) { return df_fast_two_sum(a.hi, a.lo); }
// the standard fma overloads stay visible next to the double-float one inside this namespace
using ::fma;
QXD_DF_HD dfl fma(dfl a, dfl b, dfl c) { return a * b + c; }

QXD_DF_HD double to_double(dfl a) { return (double)a.hi + (double)a.lo; }

}  // namespace qxd
