// Double-float ("df64") arithmetic on the FP32 pipes, for the high-precision parts of the
// mixed-precision step (the polish of each root and the source terms that set each
// substep's length).
//
// A value is the unevaluated sum hi + lo of two FP32 numbers with |lo| <= ulp(hi)/2:
// about 44-48 significant bits (relative rounding 4e-15 to 6e-14 per operation; FP64's
// is 1.1e-16) over FP32's exponent range.  On a GB300 one FP64 operation takes as much
// of its pipe as ~75 FP32 operations take of theirs (measured FP64 FMA rate ~1 TFLOP/s
// against ~77 TFLOP/s FP32), so an operation of ~10 FP32 instructions is several times
// cheaper than its FP64 counterpart; the step's FP64 work is dominated by exp and
// division, which gain most.
//
// Methods (published, restated here):
//  - error-free transformations: Knuth's TwoSum, Dekker's fast two-sum (|a| >= |b|), and
//    the exact product error by a fused multiply-add (Dekker's product, FMA form);
//  - addition and multiplication in the "sloppy" double-double forms of Hida, Li and
//    Bailey (2001): one error-free transformation on the leading parts, the trailing
//    parts added in plain arithmetic, one renormalisation;
//  - division by long division: q1 = a/b in FP32, the remainder a - b q1 in df64, a
//    second FP32 quotient of the remainder (FP32 quotients good to 2 units in the last
//    place, as the fast-math build's divide, give ~2^-44);
//  - square root by one Newton correction of the FP32 root;
//  - exp by Cody-Waite argument reduction x = k ln2/64 + r (ln2/64 in three FP32 pieces,
//    the first with 9 significant bits so that k times it is exact), 2^(j/64) from a
//    64-entry table of df64 values (j = k mod 64), and the Taylor series of exp(r) - 1
//    to r^5 for |r| <= ln2/128 (truncation error below 4e-17), of which only r + r^2/2
//    needs df64;
//  - log by one correction of the FP32 logarithm y0 of the mantissa m in [1, 2)
//    (x = 2^e m): with d = m exp(-y0) - 1 (small), log x = e ln2 + y0 + log(1 + d)
//    = e ln2 + y0 + d - d^2/2 + d^3/3 (error ~d^4/4, below 1e-19).
// In the fast-math build FP32 subnormals flush to zero, so a df64 value below ~2e-31
// keeps only its leading part (FP32 precision): the trailing part is ~2^-24 of it.
// Infinities would turn the trailing parts into NaN (inf - inf in the error-free
// transformations), so the type saturates instead: a conversion from FP64 maps
// magnitudes above 1e36 (and infinities) to +-1e36, exp returns 0 below -87 (FP32's
// range, flushed to zero) and exp(80) above 80, and log(0) returns -1e36.  Values that
// large or small only enter the step's terms where the FP64 result is 0 or saturated
// too (no CO formation, an infinite velocity-gradient column), and there they change
// the result by less than 1e-30 relative.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#ifndef TCG_FN
#define TCG_FN __host__ __device__ __forceinline__
#endif

namespace tcg {

// ------------------------------------------------------------------ FP32 primitives
// On the device these are written as PTX instructions without the .ftz modifier: the
// mixed kernels are built with flush-to-zero for their FP32 arithmetic, which would
// flush every trailing part below 2^-126 (those of values below ~2e-31) and the
// constants that small.  Written out, they keep subnormals, are never contracted or
// reassociated, and df64 keeps its precision down to FP32's subnormal range.  On the
// host the library is compiled without floating-point contraction or flushing.
TCG_FN float df_add_rn(float a, float b) {
#ifdef __CUDA_ARCH__
  float r;
  asm("add.rn.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
  return r;
#else
  return a + b;
#endif
}
TCG_FN float df_sub_rn(float a, float b) {
#ifdef __CUDA_ARCH__
  float r;
  asm("sub.rn.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
  return r;
#else
  return a - b;
#endif
}
TCG_FN float df_mul_rn(float a, float b) {
#ifdef __CUDA_ARCH__
  float r;
  asm("mul.rn.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
  return r;
#else
  return a * b;
#endif
}
TCG_FN float df_fma(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  float r;
  asm("fma.rn.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
#else
  return fmaf(a, b, c);
#endif
}
TCG_FN float df_neg(float a) {
#ifdef __CUDA_ARCH__
  float r;
  asm("neg.f32 %0, %1;" : "=f"(r) : "f"(a));
  return r;
#else
  return -a;
#endif
}
// FP32 quotient good to 2 units in the last place over the full range, subnormal
// operands included (a quotient digit of the df64 division).
TCG_FN float df_div(float a, float b) {
#ifdef __CUDA_ARCH__
  float r;
  asm("div.full.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
  return r;
#else
  return a / b;
#endif
}
// Correctly rounded FP32 reciprocal and an approximate square root, subnormals kept.
TCG_FN float df_rcp(float a) {
#ifdef __CUDA_ARCH__
  float r;
  asm("rcp.rn.f32 %0, %1;" : "=f"(r) : "f"(a));
  return r;
#else
  return 1.0f / a;
#endif
}
TCG_FN float df_sqrt_approx(float a) {
#ifdef __CUDA_ARCH__
  float r;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(a));
  return r;
#else
  return sqrtf(a);
#endif
}
// FP64 <-> FP32 conversions that keep subnormal FP32 values.
TCG_FN float df_f64_to_f32(double x) {
#ifdef __CUDA_ARCH__
  float r;
  asm("cvt.rn.f32.f64 %0, %1;" : "=f"(r) : "d"(x));
  return r;
#else
  return float(x);
#endif
}
TCG_FN double df_f32_to_f64(float x) {
#ifdef __CUDA_ARCH__
  double r;
  asm("cvt.f64.f32 %0, %1;" : "=d"(r) : "f"(x));
  return r;
#else
  return double(x);
#endif
}
// 2^m for -126 <= m <= 127.
TCG_FN float df_pow2i(int m) {
#ifdef __CUDA_ARCH__
  return __int_as_float((m + 127) << 23);
#else
  return ldexpf(1.0f, m);
#endif
}

// s + e = a + b exactly (Knuth).
TCG_FN void two_sum(float a, float b, float& s, float& e) {
  s = df_add_rn(a, b);
  const float bb = df_sub_rn(s, a);
  e = df_add_rn(df_sub_rn(a, df_sub_rn(s, bb)), df_sub_rn(b, bb));
}
// s + e = a + b exactly when |a| >= |b| (Dekker).
TCG_FN void fast_two_sum(float a, float b, float& s, float& e) {
  s = df_add_rn(a, b);
  e = df_sub_rn(b, df_sub_rn(s, a));
}
// p + e = a b exactly (barring underflow).
TCG_FN void two_prod(float a, float b, float& p, float& e) {
  p = df_mul_rn(a, b);
  e = df_fma(a, b, -p);
}

// ------------------------------------------------------------------ the type
constexpr double DF_BIG = 1e36;

struct df64 {
  float hi, lo;
  df64() = default;
  // From FP64: the leading 48 bits, split exactly; magnitudes above DF_BIG saturate.
  // For constants (evaluated at compile time); values computed at run time convert
  // with to_df64, which keeps subnormal trailing parts on the device.
  TCG_FN constexpr df64(double x)
      : hi((x > DF_BIG) ? float(DF_BIG) : (x < -DF_BIG) ? float(-DF_BIG) : float(x)),
        lo((x > DF_BIG || x < -DF_BIG) ? 0.0f : float(x - double(float(x)))) {}
  TCG_FN static df64 make(float h, float l) {
    df64 r;
    r.hi = h;
    r.lo = l;
    return r;
  }
  TCG_FN explicit operator double() const { return df_f32_to_f64(hi) + df_f32_to_f64(lo); }
};

// Run-time conversion from FP64 (same result as the constructor, subnormals kept).
TCG_FN df64 to_df64(double x) {
  if (x > DF_BIG) return df64::make(float(DF_BIG), 0.0f);
  if (x < -DF_BIG) return df64::make(float(-DF_BIG), 0.0f);
  const float h = df_f64_to_f32(x);
  return df64::make(h, df_f64_to_f32(x - df_f32_to_f64(h)));
}

TCG_FN df64 operator-(df64 a) { return df64::make(df_neg(a.hi), df_neg(a.lo)); }

// Out of line, like the divide and the square root: the mixed kernels are bound by
// instruction fetch, and one shared copy of the addition keeps their code smaller
// (mixed step on the 128^3 slab 57.8 -> 56.1 ms; the multiplication out of line too:
// 58.6 ms).
__host__ __device__ __noinline__ inline df64 operator+(df64 a, df64 b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = df_add_rn(e, df_add_rn(a.lo, b.lo));
  float h, l;
  fast_two_sum(s, e, h, l);
  return df64::make(h, l);
}
TCG_FN df64 operator-(df64 a, df64 b) { return a + (-b); }

TCG_FN df64 operator*(df64 a, df64 b) {
  float p, e;
  two_prod(a.hi, b.hi, p, e);
  e = df_fma(a.hi, b.lo, e);
  e = df_fma(a.lo, b.hi, e);
  float h, l;
  fast_two_sum(p, e, h, l);
  return df64::make(h, l);
}
// df64 times an FP32 number
TCG_FN df64 mul_f(df64 a, float b) {
  float p, e;
  two_prod(a.hi, b, p, e);
  e = df_fma(a.lo, b, e);
  float h, l;
  fast_two_sum(p, e, h, l);
  return df64::make(h, l);
}
// df64 plus an FP32 number
TCG_FN df64 add_f(df64 a, float b) {
  float s, e;
  two_sum(a.hi, b, s, e);
  e = df_add_rn(e, a.lo);
  float h, l;
  fast_two_sum(s, e, h, l);
  return df64::make(h, l);
}

// The quotients are FP32 divisions, not products with a reciprocal: the reciprocal of
// a subnormal divisor overflows, and 0 times it would give NaN where the quotient is 0.
__host__ __device__ __noinline__ inline df64 operator/(df64 a, df64 b) {
  const float q1 = df_div(a.hi, b.hi);
  const df64 r = a - mul_f(b, q1);  // the remainder, ~2^-22 of a
  const float q2 = df_div(r.hi, b.hi);
  float h, l;
  fast_two_sum(q1, q2, h, l);
  return df64::make(h, l);
}

TCG_FN df64& operator+=(df64& a, df64 b) { a = a + b; return a; }
TCG_FN df64& operator-=(df64& a, df64 b) { a = a - b; return a; }
TCG_FN df64& operator*=(df64& a, df64 b) { a = a * b; return a; }

TCG_FN bool operator<(df64 a, df64 b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
TCG_FN bool operator>(df64 a, df64 b) { return b < a; }
TCG_FN bool operator<=(df64 a, df64 b) { return a.hi < b.hi || (a.hi == b.hi && a.lo <= b.lo); }
TCG_FN bool operator>=(df64 a, df64 b) { return b <= a; }
TCG_FN bool operator==(df64 a, df64 b) { return a.hi == b.hi && a.lo == b.lo; }
TCG_FN bool operator!=(df64 a, df64 b) { return !(a == b); }

// ------------------------------------------------------------------ functions
TCG_FN df64 m_abs(df64 a) { return (a.hi < 0.0f) ? -a : a; }
TCG_FN df64 m_max(df64 a, df64 b) { return (a < b) ? b : a; }
TCG_FN df64 m_min(df64 a, df64 b) { return (b < a) ? b : a; }

__host__ __device__ __noinline__ inline df64 m_sqrt(df64 a) {
  if (!(a.hi > 0.0f)) return df64::make(sqrtf(a.hi), 0.0f);  // 0, or NaN below 0
  const float s = df_sqrt_approx(a.hi);
  float p, e;
  two_prod(s, s, p, e);
  // (a - s^2) / (2 s) with a - s^2 formed exactly to first order (a.hi - p is exact)
  const float r = df_add_rn(df_sub_rn(df_sub_rn(a.hi, p), e), a.lo);
  const float c = df_mul_rn(r, df_mul_rn(0.5f, df_rcp(s)));
  float h, l;
  fast_two_sum(s, c, h, l);
  return df64::make(h, l);
}

// 2^(j/64), j = 0..63 (values of the mathematical constants to 17 digits), split into
// leading and trailing FP32 parts at compile time.
#define TCG_DF_EXP2(v) {float(v), float((v) - double(float(v)))}
#define TCG_DF_EXP2_TABLE \
  {TCG_DF_EXP2(1.0), TCG_DF_EXP2(1.0108892860517005), TCG_DF_EXP2(1.0218971486541166), \
   TCG_DF_EXP2(1.0330248790212284), TCG_DF_EXP2(1.0442737824274138), TCG_DF_EXP2(1.0556451783605572), \
   TCG_DF_EXP2(1.0671404006768237), TCG_DF_EXP2(1.0787607977571199), TCG_DF_EXP2(1.0905077326652577), \
   TCG_DF_EXP2(1.1023825833078409), TCG_DF_EXP2(1.1143867425958924), TCG_DF_EXP2(1.1265216186082418), \
   TCG_DF_EXP2(1.1387886347566916), TCG_DF_EXP2(1.1511892299529827), TCG_DF_EXP2(1.1637248587775775), \
   TCG_DF_EXP2(1.1763969916502812), TCG_DF_EXP2(1.189207115002721), TCG_DF_EXP2(1.2021567314527031), \
   TCG_DF_EXP2(1.215247359980469), TCG_DF_EXP2(1.22848053610687), TCG_DF_EXP2(1.241857812073484), \
   TCG_DF_EXP2(1.2553807570246911), TCG_DF_EXP2(1.2690509571917332), TCG_DF_EXP2(1.2828700160787783), \
   TCG_DF_EXP2(1.2968395546510096), TCG_DF_EXP2(1.3109612115247644), TCG_DF_EXP2(1.3252366431597413), \
   TCG_DF_EXP2(1.3396675240533029), TCG_DF_EXP2(1.3542555469368927), TCG_DF_EXP2(1.3690024229745905), \
   TCG_DF_EXP2(1.383909881963832), TCG_DF_EXP2(1.3989796725383112), TCG_DF_EXP2(1.4142135623730951), \
   TCG_DF_EXP2(1.42961333839197), TCG_DF_EXP2(1.4451808069770467), TCG_DF_EXP2(1.460917794180647), \
   TCG_DF_EXP2(1.4768261459394993), TCG_DF_EXP2(1.4929077282912648), TCG_DF_EXP2(1.5091644275934228), \
   TCG_DF_EXP2(1.5255981507445384), TCG_DF_EXP2(1.5422108254079407), TCG_DF_EXP2(1.5590044002378369), \
   TCG_DF_EXP2(1.5759808451078865), TCG_DF_EXP2(1.593142151342267), TCG_DF_EXP2(1.6104903319492543), \
   TCG_DF_EXP2(1.6280274218573478), TCG_DF_EXP2(1.6457554781539649), TCG_DF_EXP2(1.6636765803267364), \
   TCG_DF_EXP2(1.681792830507429), TCG_DF_EXP2(1.7001063537185235), TCG_DF_EXP2(1.7186192981224779), \
   TCG_DF_EXP2(1.7373338352737062), TCG_DF_EXP2(1.7562521603732995), TCG_DF_EXP2(1.7753764925265212), \
   TCG_DF_EXP2(1.7947090750031072), TCG_DF_EXP2(1.8142521755003989), TCG_DF_EXP2(1.8340080864093424), \
   TCG_DF_EXP2(1.8539791250833855), TCG_DF_EXP2(1.8741676341103), TCG_DF_EXP2(1.8945759815869656), \
   TCG_DF_EXP2(1.9152065613971474), TCG_DF_EXP2(1.9360617934922943), TCG_DF_EXP2(1.9571441241754002), \
   TCG_DF_EXP2(1.9784560263879509)}
static __device__ const float2 kDfExp2Dev[64] = TCG_DF_EXP2_TABLE;
static const float2 kDfExp2Host[64] = TCG_DF_EXP2_TABLE;

// exp(x) for a df64 argument (method in the header comment).
__host__ __device__ __noinline__ inline df64 m_exp(df64 x) {
  if (x.hi < -87.0f) return df64::make(0.0f, 0.0f);
  if (x.hi > 80.0f) x = df64::make(80.0f, 0.0f);
  if (!(x.hi == x.hi)) return x;  // NaN
  // ln2/64 = C1 + C2 + C3 (C1 = 0x1.63p-7, 9 significant bits: k C1 is exact for |k| < 2^15)
  constexpr float C1 = 0.0108337402343750f;
  constexpr float C2 = -3.3155382e-06f;
  constexpr float C3 = 2.5728046e-14f;
  constexpr float INV = 92.33248261689366f;  // 64 / ln 2
  const float kf = rintf(x.hi * INV);
  const int k = (int)kf;
  // r = x - k ln2/64: x.hi - k C1 is exact (k C1 is exact, and within a factor 2 of x.hi)
  const float a = df_sub_rn(x.hi, df_mul_rn(kf, C1));
  df64 r;
  {
    float s, e;
    two_sum(a, x.lo, s, e);
    float p, pe;
    two_prod(kf, C2, p, pe);
    float s2, e2;
    two_sum(s, -p, s2, e2);
    e = df_add_rn(df_add_rn(e, e2), df_sub_rn(-pe, df_mul_rn(kf, C3)));
    float h, l;
    fast_two_sum(s2, e, h, l);
    r = df64::make(h, l);
  }
  // exp(r) - 1 = r + r^2/2 + r^3 (1/6 + r/24 + r^2/120) for |r| <= ln2/128: r^2/2 in df64
  // (its square exact from Dekker's product), the cubic group (below 3e-8) in FP32
  df64 em1;
  {
    float p, pe;
    two_prod(r.hi, r.hi, p, pe);
    pe = df_fma(2.0f * r.hi, r.lo, pe);
    float h, l;
    fast_two_sum(df_mul_rn(0.5f, p), df_mul_rn(0.5f, pe), h, l);
    em1 = r + df64::make(h, l);
    const float rh = r.hi;
    float q = df_fma(rh, 1.0f / 120.0f, 1.0f / 24.0f);
    q = df_fma(rh, q, 1.0f / 6.0f);
    q = df_mul_rn(df_mul_rn(df_mul_rn(rh, rh), rh), q);
    em1 = add_f(em1, q);
  }
  // exp(x) = 2^m 2^(j/64) (1 + em1) with k = 64 m + j
  const int j = k & 63;
  const int m = (k - j) / 64;
#ifdef __CUDA_ARCH__
  const float2 t = __ldg(&kDfExp2Dev[j]);
#else
  const float2 t = kDfExp2Host[j];
#endif
  const df64 tj = df64::make(t.x, t.y);
  const df64 y = tj + tj * em1;
  const float sc = df_pow2i(m);
  return df64::make(df_mul_rn(y.hi, sc), df_mul_rn(y.lo, sc));
}

// log(x) for a df64 argument (method in the header comment), with x first scaled by a
// power of two into [1, 2): x = 2^e m, log x = e ln2 + log m.  Then exp(-y0) stays in
// (1/2, 1], far from the flush-to-zero range, for any x.
__host__ __device__ __noinline__ inline df64 m_log(df64 x) {
  if (!(x.hi > 0.0f)) {
    if (x.hi == 0.0f) return df64::make(float(-DF_BIG), 0.0f);
    return df64::make(logf(x.hi), 0.0f);  // NaN
  }
  int ex;
  (void)frexpf(x.hi, &ex);  // x.hi = f 2^ex, f in [1/2, 1)
  int e = ex - 1;
  if (e > 126) e = 126;
  if (e < -126) e = -126;
  const float sc = df_pow2i(-e);
  const df64 m = df64::make(df_mul_rn(x.hi, sc), df_mul_rn(x.lo, sc));
  const float y0 = logf(m.hi);
  const df64 d = add_f(m * m_exp(df64::make(-y0, 0.0f)), -1.0f);
  const float dh = d.hi;
  const float corr = df_mul_rn(df_mul_rn(dh, dh), df_fma(dh, 1.0f / 3.0f, -0.5f));
  // e ln2 with ln2 = L1 + L2 + L3 (L1 = 0x1.62e4p-1, 16 significant bits: e L1 is exact)
  constexpr float L1 = 0.693145751953125f, L2 = 1.4286068e-06f, L3 = 5.497923e-14f;
  const float fe = float(e);
  float p, pe;
  two_prod(fe, L2, p, pe);
  df64 eln2;
  {
    float s1, e1;
    two_sum(df_mul_rn(fe, L1), p, s1, e1);
    e1 = df_add_rn(e1, df_add_rn(pe, df_mul_rn(fe, L3)));
    float h, l;
    fast_two_sum(s1, e1, h, l);
    eln2 = df64::make(h, l);
  }
  return add_f(eln2 + (df64::make(y0, 0.0f) + d), corr);
}

}  // namespace tcg
