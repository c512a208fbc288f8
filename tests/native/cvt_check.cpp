// Host check of the integer-pipe binary32 <-> binary64 conversions of
// cvt.cuh against the host's own conversions (IEEE 754 round to nearest
// even): every binary32 value for the widening, and seeded random binary64
// values of every exponent plus the rounding and range boundaries for the
// narrowing.  Prints one line per failure (at most 20) and "ok <counts>".
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "../../paper_2011_01316_gb300/csrc/cvt.cuh"

using namespace expdg;

static uint64_t dbits(double x) {
  uint64_t u;
  std::memcpy(&u, &x, 8);
  return u;
}
static double dfrom(uint64_t u) {
  double x;
  std::memcpy(&x, &u, 8);
  return x;
}

static uint64_t state = 0x9e3779b97f4a7c15ull;
static uint64_t next() {  // splitmix64
  uint64_t z = (state += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

int main(int argc, char** argv) {
  long fails = 0;
  // widening: every binary32 bit pattern
  uint64_t n32 = 0;
  for (uint64_t u = 0; u <= 0xffffffffull; ++u) {
    float f;
    const uint32_t b = (uint32_t)u;
    std::memcpy(&f, &b, 4);
    const double got = f32_to_f64_exact(f), ref = (double)f;
    const bool ok = std::isnan(ref) ? (std::isnan(got) && (dbits(got) >> 63) == (b >> 31)) : dbits(got) == dbits(ref);
    if (!ok && fails++ < 20) std::printf("widen %08x: got %016llx ref %016llx\n", b, (unsigned long long)dbits(got),
                                        (unsigned long long)dbits(ref));
    ++n32;
  }
  // narrowing: random patterns (uniform over bits, hence over exponents), then
  // values near the rounding midpoints and the range ends
  const long nrand = argc > 1 ? std::atol(argv[1]) : 20000000;
  uint64_t n64 = 0;
  auto check = [&](double x) {
    const float got = f64_to_f32_rn(x), ref = (float)x;
    uint32_t gb, rb;
    std::memcpy(&gb, &got, 4);
    std::memcpy(&rb, &ref, 4);
    const bool ok = std::isnan(ref) ? std::isnan(got) : gb == rb;
    if (!ok && fails++ < 20)
      std::printf("narrow %016llx (%.17g): got %08x ref %08x\n", (unsigned long long)dbits(x), x, gb, rb);
    ++n64;
  };
  for (long k = 0; k < nrand; ++k) check(dfrom(next()));
  for (int e = 860; e <= 1160; ++e)  // every exponent around the binary32 range
    for (int k = 0; k < 20000; ++k) {
      const uint64_t r = next();
      uint64_t frac = r & 0x000fffffffffffffull;
      const int mode = k % 4;  // exact midpoints, one ulp either side, random
      if (mode != 3) frac = (frac & ~0x1fffffffull) | 0x10000000ull;
      if (mode == 1) frac += 1;
      if (mode == 2) frac -= 1;
      check(dfrom(((uint64_t)(r >> 63) << 63) | ((uint64_t)e << 52) | frac));
    }
  const double specials[] = {0.0, -0.0, INFINITY, -INFINITY, NAN, 3.4028234663852886e38, 3.4028235677973366e38,
                             3.4028235677973362e38, 1.1754943508222875e-38, 1.401298464324817e-45,
                             7.006492321624085e-46, 7.006492321624087e-46, 2.1019476964872256e-45, 1e-300, 1e300,
                             4.9e-324};
  for (double x : specials) {
    check(x);
    check(-x);
  }
  std::printf("%s widened %llu narrowed %llu failures %ld\n", fails ? "FAIL" : "ok", (unsigned long long)n32,
              (unsigned long long)n64, fails);
  return fails ? 1 : 0;
}
