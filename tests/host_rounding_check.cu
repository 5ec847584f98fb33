// Host-side check of the roundings the update kernel uses for X <- RN(X1 + U) (Alg. 1's update):
// add_on_grid_rn (the usual case, on x1's grid) and add_exact_rn (exact 128-bit sum), compiled
// as host code from the library's own header.  Random, tie and binade-edge inputs, x1 near the
// bottom of the normal range and x1 = 0 among them; where both succeed their bits must agree.
// Results of either form are written out (up to MAXDUMP of each, tagged G and E) so that the
// test can check them against exact rational rounding; a form that cannot give a normal result
// must decline (the kernel then takes its general path), which that check also covers.
//
// usage: host_rounding_check CASES SEED DUMPFILE MAXDUMP
#include <cstdio>
#include <cstdlib>
#include <random>

#include "intround.cuh"

using namespace frx;

int main(int argc, char** argv) {
  if (argc != 5) {
    std::fprintf(stderr, "usage: %s CASES SEED DUMPFILE MAXDUMP\n", argv[0]);
    return 2;
  }
  const long long cases = std::atoll(argv[1]);
  std::mt19937_64 g(std::strtoull(argv[2], nullptr, 10));
  FILE* df = std::fopen(argv[3], "w");
  const long long maxdump = std::atoll(argv[4]);
  if (!df) return 2;
  long long grid = 0, exact = 0, both = 0, mismatches = 0, dumped = 0, dumped_e = 0, ties = 0, tiny = 0;
  for (long long it = 0; it < cases; ++it) {
    // x1: random sign, binade in [-20, 5] (one case in eight: in [-1022, -990], next to the
    // subnormal range; one in sixteen: x1 = 0); some exact powers of two and values next to them
    u64 mant = g() & ((1ull << 52) - 1);
    const int kind = (int)(g() % 8);
    if (kind == 0) mant = 0;
    if (kind == 1) mant = (1ull << 52) - 1 - g() % 4;
    if (kind == 2) mant = g() % 4;
    const int range = (int)(g() % 16);
    const int e = range < 2 ? -1022 + (int)(g() % 33) : (int)(g() % 26) - 20;
    if (range < 2) ++tiny;
    u64 b = ((u64)(e + 1023) << 52) | mant | ((g() & 1) ? (1ull << 63) : 0ull);
    if (range == 2) b &= 1ull << 63;   // signed zero
    const double x1 = bits_to_double(b);
    // N: up to 118 bits, either sign; s = q - c from -6 to 133 (q = e - 52, x1's ulp exponent)
    const int w = 1 + (int)(g() % 118);
    u128 mag = ((u128)g() << 64) | (u128)g();
    mag &= (((u128)1) << w) - 1;
    i128 N = (g() & 1) ? -(i128)mag : (i128)mag;
    const int s = (int)(g() % 140) - 6;
    if (g() % 4 == 0 && s >= 1 && s < 120) {   // an exact tie: bit s-1 set, nothing below
      N &= ~((((i128)1) << s) - 1);
      N |= ((i128)1) << (s - 1);
      if (g() & 1) N = -N;
      ++ties;
    }
    const int c = (e - 52) - s;
    double r1 = 0.0, r2 = 0.0;
    const bool ok1 = add_on_grid_rn(x1, N, c, r1);
    const bool ok2 = add_exact_rn(x1, N, c, r2);
    if (ok1) {
      ++grid;
      if (dumped < maxdump) {
        std::fprintf(df, "G %016llx %d %016llx %016llx %016llx\n", (unsigned long long)b, c,
                     (unsigned long long)((u128)N >> 64), (unsigned long long)(u64)N,
                     (unsigned long long)double_to_bits(r1));
        ++dumped;
      }
      if (ok2) {
        ++both;
        if (double_to_bits(r1) != double_to_bits(r2)) ++mismatches;
      }
    }
    if (ok2) {
      ++exact;
      // the exact form's own results: every one near the bottom of the range, a sample elsewhere
      if (dumped_e < maxdump && (range < 3 || g() % 8 == 0)) {
        std::fprintf(df, "E %016llx %d %016llx %016llx %016llx\n", (unsigned long long)b, c,
                     (unsigned long long)((u128)N >> 64), (unsigned long long)(u64)N,
                     (unsigned long long)double_to_bits(r2));
        ++dumped_e;
      }
    }
  }
  std::fclose(df);
  std::printf("cases %lld ties %lld tiny %lld grid %lld exact %lld both %lld mismatches %lld dumped %lld "
              "dumped_e %lld\n", cases, ties, tiny, grid, exact, both, mismatches, dumped, dumped_e);
  return mismatches != 0;
}
