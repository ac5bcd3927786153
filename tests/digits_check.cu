// Host check of the exact-digit arithmetic of the tensor-core Gram matrix
// (tc_common.cuh digit_step and the class-sum windows of gram_tc.cu): values
// on a per-column power-of-two grid cut into BF16 digits, every digit an
// integer of at most 8 significant bits, the reconstruction exact; class sums
// of a 128-row window (the longest the kernel accumulates) below 2^24 at every
// partial sum, so an FP32 accumulator holds them exactly; and the whole
// estimate of X^T X (classes folded into FP32 pairs, the pairs flushed into
// FP64 every 8 windows, as the kernel's epilogue does) against long double.  Prints name/value pairs for
// tests/test_gram_digits_host.py.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

#include "df32.cuh"
#include "tc_common.cuh"

typedef long double LD;

static uint64_t g_state = 0x243F6A8885A308D3ull;
static double urand() {  // xorshift64*, uniform in [0, 1)
  g_state ^= g_state >> 12;
  g_state ^= g_state << 25;
  g_state ^= g_state >> 27;
  return (double)((g_state * 0x2545F4914F6CDD1Dull) >> 11) * 0x1p-53;
}
static double nrand() {  // Box-Muller
  const double u1 = 1.0 - urand(), u2 = urand();
  return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
}
static bool is_bf16_exact(float d) {  // an integer of at most 8 significant bits
  if (d != std::rint(d)) return false;
  float a = std::fabs(d);
  if (a == 0.0f) return true;
  while (a >= 256.0f && std::fmod(a, 2.0f) == 0.0f) a *= 0.5f;
  return a <= 256.0f;
}

static float to_bf16(float x) {  // round to nearest even BF16
  uint32_t b;
  std::memcpy(&b, &x, 4);
  b += 0x7FFFu + ((b >> 16) & 1u);
  b &= 0xFFFF0000u;
  float y;
  std::memcpy(&y, &b, 4);
  return y;
}

// S digits; all_pairs: every digit pair (else t + u <= S + 1); bf16: data rounded to BF16.
static void run(const char* tag, int S, bool all_pairs, bool bf16) {
  const int rows = 16384, cols = 6, win = 128;
  const int last = all_pairs ? 2 * S : S + 1;
  std::vector<float> X((size_t)rows * cols);
  int E[cols];
  for (int j = 0; j < cols; ++j) {
    float m = 0.0f;
    for (int r = 0; r < rows; ++r) {
      // column scales 2^-20 .. 2^20 and a few tiny and exactly-zero entries
      float x = (float)(nrand() * std::ldexp(1.0, 8 * j - 20));
      if (r % 97 == 3) x *= 1e-9f;
      if (r % 131 == 5) x = 0.0f;
      if (bf16) x = to_bf16(x);
      X[(size_t)r * cols + j] = x;
      m = std::fmax(m, std::fabs(x));
    }
    std::frexp(m, &E[j]);
  }
  // digits
  int exact = 1, bounds = 1;
  double max_rest = 0.0;
  std::vector<float> D((size_t)rows * cols * S);
  for (int r = 0; r < rows; ++r)
    for (int j = 0; j < cols; ++j) {
      const float v = std::ldexp(X[(size_t)r * cols + j], -E[j]);
      float rr = v;
      LD recon = 0.0L;
      for (int t = 0; t < S; ++t) {
        const float d = hs::tc::digit_step(rr);
        D[((size_t)r * cols + j) * S + t] = d;
        exact &= is_bf16_exact(d);
        bounds &= (std::fabs(d) <= (t == 0 ? 256.0f : 128.0f));
        recon += std::ldexp((LD)d, -8 * (t + 1));
      }
      exact &= (recon + std::ldexp((LD)rr, -8 * S) == (LD)v);  // v = sum of digits + rest, exactly
      max_rest = std::fmax(max_rest, (double)std::fabs((LD)v - recon) * std::ldexp(1.0, 8 * S));
    }
  // class sums per window; FP32 running sums checked against the exact integers
  int window_exact = 1;
  double class_max = 0.0;
  double gram_err = 0.0;
  for (int i = 0; i < cols; ++i)
    for (int j = 0; j <= i; ++j) {
      float ah = 0.0f, al = 0.0f;  // the epilogue's pair accumulator
      double acc = 0.0;            // its FP64 accumulator (flushed every 8 windows)
      for (int r0 = 0; r0 < rows; r0 += win) {
        float c[16];
        for (int w = 2; w <= last; ++w) {
          float f = 0.0f;
          int64_t ex = 0;
          for (int r = r0; r < r0 + win; ++r)
            for (int t = 1; t <= S; ++t) {
              const int u = w - t;
              if (u < 1 || u > S) continue;
              const float a = D[((size_t)r * cols + i) * S + t - 1], b = D[((size_t)r * cols + j) * S + u - 1];
              f += a * b;
              ex += (int64_t)a * (int64_t)b;
              class_max = std::fmax(class_max, std::fabs((double)ex));
              window_exact &= ((double)f == (double)ex);
            }
          c[w] = f;
        }
        // f = sum_w C_w 2^{-8(w-2)} by Horner from the smallest class, in pairs
        float fh = c[last], fl = 0.0f;
        for (int w = last - 1; w >= 2; --w) {
          const float a = fh * 0x1p-8f, b = c[w];
          const float sum = a + b, bb = sum - a;
          const float e2 = (a - (sum - bb)) + (b - bb);
          fh = sum;
          fl = std::fma(fl, 0x1p-8f, e2);
        }
        const hs::df2 v = hs::df_add(hs::df2{ah, al}, hs::df2{fh, fl});
        ah = v.hi;
        al = v.lo;
        if ((r0 / win + 1) % 8 == 0) {
          acc += (double)ah + (double)al;
          ah = al = 0.0f;
        }
      }
      const LD got = std::ldexp(((LD)acc + ((LD)ah + (LD)al)) * 0x1p-16L, E[i] + E[j]);
      LD ref = 0.0L, nrm = 0.0L;
      for (int r = 0; r < rows; ++r) {
        ref += (LD)X[(size_t)r * cols + i] * (LD)X[(size_t)r * cols + j];
        nrm += std::fabs((LD)X[(size_t)r * cols + i] * (LD)X[(size_t)r * cols + j]);
      }
      gram_err = std::fmax(gram_err, (double)(std::fabs(got - ref) / nrm));
    }
  std::printf("%s_digits_exact %d %s_digit_bounds %d %s_rest %.3e %s_window_exact %d %s_class_max %.6e %s_gram_err %.3e\n",
              tag, exact, tag, bounds, tag, max_rest, tag, window_exact, tag, class_max, tag, gram_err);
}

int main() {
  run("f32", 5, false, false);   // FP32 X: five digits, pairs with t + u <= 6
  run("bf16", 4, true, true);    // BF16 X: four digits, every pair
  return 0;
}
