// Host check of the FP32-pair arithmetic the factorization uses (df32.cuh):
// random operands, each result compared with long double arithmetic.  Prints
// the largest error of each operation, relative to the exact result (for the
// sum, to |a| + |b|; for the 32-term dot products, to the sum of |a_q b_q|), for
// tests/test_df32_host.py.
#include <cmath>
#include <cstdint>
#include <cstdio>

#include "df32.cuh"

using hs::df2;
typedef long double LD;

static uint64_t g_state = 0x9E3779B97F4A7C15ull;
static double urand() {  // xorshift64*, uniform in [0, 1)
  g_state ^= g_state >> 12;
  g_state ^= g_state << 25;
  g_state ^= g_state >> 27;
  return (double)((g_state * 0x2545F4914F6CDD1Dull) >> 11) * 0x1p-53;
}
static double rval() {  // sign * 2^U(-8, 8) * U[1, 2)
  const double m = 1.0 + urand(), e = std::floor(urand() * 16.0) - 8.0;
  return (urand() < 0.5 ? -1.0 : 1.0) * std::ldexp(m, (int)e);
}
static LD val(df2 a) { return (LD)a.hi + (LD)a.lo; }

int main() {
  double e_add = 0, e_mul = 0, e_rec = 0, e_sqrt = 0, e_dot = 0, e_split = 0;
  for (int it = 0; it < 200000; ++it) {
    const double x = rval(), y = rval();
    const df2 a = hs::df_split(x), b = hs::df_split(y);
    const LD A = val(a), B = val(b);
    e_split = std::fmax(e_split, (double)std::fabs((val(a) - (LD)x) / (LD)x));
    // pair addition: error relative to |a| + |b| (the sum may cancel)
    e_add = std::fmax(e_add, (double)(std::fabs(val(hs::df_add(a, b)) - (A + B)) / (std::fabs(A) + std::fabs(B))));
    e_mul = std::fmax(e_mul, (double)std::fabs((val(hs::df_mul(a, b)) - A * B) / (A * B)));
    e_rec = std::fmax(e_rec, (double)std::fabs((val(hs::df_recip(b)) - 1.0L / B) * B));
    const LD aa = std::fabs(A);
    const df2 sa = hs::df_sqrt(df2{std::fabs(a.hi), a.hi < 0 ? -a.lo : a.lo});
    e_sqrt = std::fmax(e_sqrt, (double)std::fabs((val(sa) - std::sqrt(aa)) / std::sqrt(aa)));
  }
  for (int it = 0; it < 20000; ++it) {
    float sh = 0.f, sl = 0.f;
    LD exact = 0, absum = 0;
    for (int q = 0; q < 32; ++q) {
      const df2 a = hs::df_split(rval()), b = hs::df_split(rval());
      hs::df_fma(sh, sl, a, b);
      exact += val(a) * val(b);
      absum += std::fabs(val(a) * val(b));
    }
    const df2 r = hs::df_renorm(sh, sl);
    e_dot = std::fmax(e_dot, (double)(std::fabs(val(r) - exact) / absum));
  }
  std::printf("split %.3e add %.3e mul %.3e recip %.3e sqrt %.3e dot32 %.3e\n", e_split, e_add, e_mul, e_rec, e_sqrt,
              e_dot);
  return 0;
}
