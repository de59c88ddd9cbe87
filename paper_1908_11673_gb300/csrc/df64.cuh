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
#include <cstring>

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

// ---- conversions between FP64 and double-float by integer operations ---------------
// On GB300 the conversions between FP64 and FP32 run on the FP64 pipe (1/64 of the FP32
// rate), which makes a pass that converts a whole field ALU-bound.  The IEEE-754 binary64
// and binary32 encodings give the same results with integer operations:
//   df_split(d) = (RN32(d), RN32(d - RN32(d)))    (the dfl(double) constructor)
//   df_widen(f) = (double)f                        (exact)
// for the ranges noted; other inputs (zero, subnormal, very large or small magnitudes,
// inf, nan) take the conversion instructions.
QXD_DF_HD unsigned long long df_bits(double d) {
#ifdef __CUDA_ARCH__
    return (unsigned long long)__double_as_longlong(d);
#else
    unsigned long long u;
    std::memcpy(&u, &d, sizeof u);
    return u;
#endif
}
QXD_DF_HD double df_double_of(unsigned long long u) {
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)u);
#else
    double d;
    std::memcpy(&d, &u, sizeof d);
    return d;
#endif
}
QXD_DF_HD unsigned df_fbits(float f) {
#ifdef __CUDA_ARCH__
    return (unsigned)__float_as_int(f);
#else
    unsigned u;
    std::memcpy(&u, &f, sizeof u);
    return u;
#endif
}
QXD_DF_HD float df_float_of(unsigned u) {
#ifdef __CUDA_ARCH__
    return __int_as_float((int)u);
#else
    float f;
    std::memcpy(&f, &u, sizeof f);
    return f;
#endif
}

// (RN32(d), RN32(d - RN32(d))).  Integer path for biased exponents 949..1149 (|d| in
// [2^-74, 2^127)): there both parts are normal floats or zero.  With M the 53-bit
// significand, the leading part is M rounded to 24 bits (to nearest, ties to even); the
// remainder d - hi = diff 2^(e - 1075) with |diff| <= 2^28, so its rounding is the
// rounding of the integer diff, scaled by a power of two.
QXD_DF_HD dfl df_split(double d) {
    const unsigned long long u = df_bits(d);
    const int e = (int)((u >> 52) & 0x7FF);
    if (e < 949 || e > 1149) return dfl(d);
    const unsigned long long M = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    unsigned long long q = M >> 29;
    const unsigned long long rem = M & 0x1FFFFFFFull;
    if (rem > 0x10000000ull || (rem == 0x10000000ull && (q & 1ull))) ++q;
    const long long diff = (long long)M - (long long)(q << 29);
    int E = e - 896;  // binary32 biased exponent
    if (q == (1ull << 24)) {  // rounding carried into the next binade
        q >>= 1;
        ++E;
    }
    const unsigned sign = (unsigned)(u >> 63);
    const float hi = df_float_of((sign << 31) | ((unsigned)E << 23) | ((unsigned)q & 0x7FFFFFu));
    const int ad = (int)(diff < 0 ? -diff : diff);
    const float scale = df_float_of((unsigned)(e - 1075 + 127) << 23);
    const float mag = QXD_FMUL((float)ad, scale);
    const bool neg = diff != 0 && ((sign != 0) != (diff < 0));  // d - hi = +0 when exact
    return dfl(hi, neg ? -mag : mag);
}

// (double)f; integer path for zero and normal floats
QXD_DF_HD double df_widen(float f) {
    const unsigned b = df_fbits(f);
    const unsigned E = (b >> 23) & 0xFFu;
    const unsigned long long s = (unsigned long long)(b >> 31) << 63;
    if ((b & 0x7FFFFFFFu) == 0) return df_double_of(s);
    if (E == 0 || E == 255) return (double)f;
    return df_double_of(s | ((unsigned long long)(E + 896) << 52) | ((unsigned long long)(b & 0x7FFFFFu) << 29));
}

}  // namespace qxd
