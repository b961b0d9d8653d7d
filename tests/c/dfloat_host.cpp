// Host build of the library's double-word arithmetic (csrc/dfloat.cuh) for
// the CPU tests.  The header is compiled as it is; the CUDA intrinsics it
// calls are given host definitions with the same IEEE semantics (single
// roundings to nearest, an exact fused multiply-add, bit reinterpretations;
// the approximate reciprocal division of the device is an exact division
// here, which only makes the Newton seed better).  Build with
// -ffp-contract=off so that the host compiler does not fuse what the device
// code keeps separate.
//
// The program draws operands with a fixed-seed generator, applies every
// operation and prints operands and results as hexadecimal floats, one case
// per line:  <op> <operands...> ; <results...>
// The Python test recomputes each result exactly (rationals) and checks the
// published error bounds.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>

static inline float __fadd_rn(float a, float b) { return a + b; }
static inline float __fsub_rn(float a, float b) { return a - b; }
static inline float __fmul_rn(float a, float b) { return a * b; }
static inline float __fmaf_rn(float a, float b, float c) { return std::fmaf(a, b, c); }
static inline float __fdividef(float a, float b) { return a / b; }
static inline float __uint2float_rn(unsigned u) { return (float)u; }
static inline float __uint_as_float(unsigned u) {
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}
static inline unsigned __float_as_uint(float f) {
  unsigned u;
  std::memcpy(&u, &f, 4);
  return u;
}
static inline long long __double_as_longlong(double d) {
  long long l;
  std::memcpy(&l, &d, 8);
  return l;
}
static inline double __longlong_as_double(long long l) {
  double d;
  std::memcpy(&d, &l, 8);
  return d;
}

#include "dfloat.cuh"

using icon::df;
using icon::dws;

static uint64_t g_state = 0x9e3779b97f4a7c15ull;
static uint64_t next_u64() {  // xorshift64*
  g_state ^= g_state >> 12;
  g_state ^= g_state << 25;
  g_state ^= g_state >> 27;
  return g_state * 0x2545f4914f6cdd1dull;
}
static double uniform() { return (double)(next_u64() >> 11) * (1.0 / 9007199254740992.0); }

// a double of either sign with a random exponent in 2^[-e, e]
static double rand_double(int e) {
  const double m = 1.0 + uniform();
  const int x = (int)(next_u64() % (uint64_t)(2 * e + 1)) - e;
  return (next_u64() & 1 ? -1.0 : 1.0) * std::ldexp(m, x);
}
static df rand_df(int e) { return icon::to_df(rand_double(e)); }

static void pr(float x) { std::printf(" %a", (double)x); }
static void prd(double x) { std::printf(" %a", x); }

int main() {
  const int n = 4000;
  for (int i = 0; i < n; ++i) {
    // error-free transformations
    const float a = (float)rand_double(20), b = (float)rand_double(20);
    const df s = icon::two_sum(a, b);
    std::printf("two_sum");
    pr(a), pr(b), std::printf(" ;"), pr(s.hi), pr(s.lo), std::printf("\n");
    const float big = std::fabs(a) >= std::fabs(b) ? a : b, small = std::fabs(a) >= std::fabs(b) ? b : a;
    const df f = icon::fast_two_sum(big, small);
    std::printf("fast_two_sum");
    pr(big), pr(small), std::printf(" ;"), pr(f.hi), pr(f.lo), std::printf("\n");
    // conversions
    const double x = rand_double(60);
    const df c = icon::to_df(x);
    std::printf("to_df");
    prd(x), std::printf(" ;"), pr(c.hi), pr(c.lo), std::printf("\n");
    std::printf("to_double");
    pr(c.hi), pr(c.lo), std::printf(" ;"), prd(icon::to_double(c)), std::printf("\n");
    std::printf("f2d_exact");
    pr(a), std::printf(" ;"), prd(icon::f2d_exact(a)), std::printf("\n");
    // double-word operations; the second operand of the additions sometimes
    // nearly cancels the first
    const df p = rand_df(10);
    df q = rand_df(10);
    if (i % 3 == 0) q = icon::to_df(-icon::to_double(p) * (1.0 + std::ldexp(uniform(), -20)));
    const df add = p + q;
    std::printf("add");
    pr(p.hi), pr(p.lo), pr(q.hi), pr(q.lo), std::printf(" ;"), pr(add.hi), pr(add.lo), std::printf("\n");
    const dws sl = dws{p.hi, p.lo} + dws{q.hi, q.lo};
    std::printf("add_sloppy");
    pr(p.hi), pr(p.lo), pr(q.hi), pr(q.lo), std::printf(" ;"), pr(sl.hi), pr(sl.lo), std::printf("\n");
    const df ps = icon::to_df(std::fabs(icon::to_double(p))), qs = icon::to_df(std::fabs(icon::to_double(q)));
    const df same = icon::add_same_sign(ps, qs);
    std::printf("add_same_sign");
    pr(ps.hi), pr(ps.lo), pr(qs.hi), pr(qs.lo), std::printf(" ;"), pr(same.hi), pr(same.lo), std::printf("\n");
    const df m = p * q;
    std::printf("mul");
    pr(p.hi), pr(p.lo), pr(q.hi), pr(q.lo), std::printf(" ;"), pr(m.hi), pr(m.lo), std::printf("\n");
    const df mf = p * b;
    std::printf("mul_fp");
    pr(p.hi), pr(p.lo), pr(b), std::printf(" ;"), pr(mf.hi), pr(mf.lo), std::printf("\n");
    const df af = p + b;
    std::printf("add_fp");
    pr(p.hi), pr(p.lo), pr(b), std::printf(" ;"), pr(af.hi), pr(af.lo), std::printf("\n");
    const df r = icon::rcp(p);
    std::printf("rcp");
    pr(p.hi), pr(p.lo), std::printf(" ;"), pr(r.hi), pr(r.lo), std::printf("\n");
  }
  // special values of the conversions
  const double specials[] = {0.0, -0.0, 1.0, -1.0, 1e-40, -1e-40, 3.0e38, 4.0e38, -4.0e38, INFINITY, -INFINITY, NAN};
  for (double x : specials) {
    const df c = icon::to_df(x);
    std::printf("to_df_special");
    prd(x), std::printf(" ;"), pr(c.hi), pr(c.lo), std::printf("\n");
  }
  return 0;
}
