// Host check of the integer-unit float operations in sor_bits.cuh against the
// host's IEEE conversions and multiplication (round to nearest, ties to even):
// random bit patterns of every class plus hand-picked boundary values.
// Prints the number of mismatches per operation; exit status 0 when all match.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <limits>
#include <random>
#include <vector>

#include "sor_bits.cuh"

using namespace sorgb;

static bool same64(double a, double b) { return bits_of(a) == bits_of(b) || (std::isnan(a) && std::isnan(b)); }
static bool same32(float a, float b) { return bits_of(a) == bits_of(b) || (std::isnan(a) && std::isnan(b)); }

int main(int argc, char** argv) {
  const long count = argc > 1 ? std::atol(argv[1]) : 2000000;
  std::mt19937_64 g(12345);
  long bad_w = 0, bad_t = 0, bad_n = 0;
  std::vector<double> d_edge = {0.0, -0.0, 1.0, -1.0, 4.0, std::numeric_limits<double>::min(),
                                std::numeric_limits<double>::denorm_min(), std::numeric_limits<double>::max(),
                                std::numeric_limits<double>::max() / 4.0, std::numeric_limits<double>::max() / 3.9,
                                std::numeric_limits<double>::infinity(), -std::numeric_limits<double>::infinity(),
                                std::numeric_limits<double>::quiet_NaN(), (double)std::numeric_limits<float>::max(),
                                (double)std::numeric_limits<float>::min(), (double)std::numeric_limits<float>::denorm_min(),
                                3.4028235677973366e38, 3.4028234663852886e38, 1.1754942807573643e-38,
                                1.1754943508222875e-38, 1.0000000596046448, 1.0000001788139343, 0.5 * 1.1754943508222875e-38};
  std::vector<float> f_edge = {0.0f, -0.0f, 1.0f, -2.5f, std::numeric_limits<float>::min(),
                               std::numeric_limits<float>::denorm_min(), std::numeric_limits<float>::max(),
                               std::numeric_limits<float>::infinity(), std::numeric_limits<float>::quiet_NaN()};
  auto check_d = [&](double x) {
    if (!same64(times4(x), x * 4.0)) ++bad_t;
    if (!same32(narrow_f64(x), (float)x)) ++bad_n;
  };
  auto check_f = [&](float x) {
    if (!same64(widen_f32(x), (double)x)) ++bad_w;
  };
  for (double x : d_edge) {
    check_d(x);
    check_d(-x);
    check_d(std::nextafter(x, 0.0));
    check_d(std::nextafter(x, INFINITY));
  }
  for (float x : f_edge) {
    check_f(x);
    check_f(-x);
  }
  for (long k = 0; k < count; ++k) {
    const uint64_t r = g();
    check_d(f64_of(r));                                          // any binary64 pattern
    uint64_t near = (r & 0x800FFFFFFFFFFFFFull) | ((uint64_t)(896 + (r >> 53) % 260) << 52);
    check_d(f64_of(near));                                       // exponents around the binary32 range
    check_d(f64_of((r & ~((1ull << 29) - 1)) | (1ull << 28)));   // exact ties for the narrowing
    check_f(f32_of((uint32_t)r));                                // any binary32 pattern
  }
  std::printf("widen %ld times4 %ld narrow %ld mismatches over %ld random values\n", bad_w, bad_t, bad_n, count);
  return (bad_w || bad_t || bad_n) ? 1 : 0;
}
