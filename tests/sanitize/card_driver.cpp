// Card expansion of the CUDA library's host side (pdr_card.h: card
// validation and expansion; pdr_hot.h: the shared-memory card image) under
// AddressSanitizer / UndefinedBehaviorSanitizer (test infrastructure).
//
// Reads pdr_card structs from the file given (raw bytes, one after another),
// expands each, then expands a few thousand mutated copies (fields set to
// out-of-range, huge, negative or non-finite values) that the validation
// must either accept or reject cleanly.  Exit status 0 when every call
// returned normally; prints the numbers of accepted and rejected cards.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <memory>
#include <vector>

#include "pdr_card.h"
#include "pdr_hot.h"

namespace pdr {
int set_last_error(int code, const char*) { return code; }
}  // namespace pdr

static uint64_t rng_state = 0x9E3779B97F4A7C15ull;
static uint64_t next() {  // splitmix64
  uint64_t z = (rng_state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static double odd_value() {
  const double v[] = {0.0, -1.0, 1e-12, 1e12, 7.0, 2.5, 4.9, 1e300,
                      std::numeric_limits<double>::quiet_NaN(), std::numeric_limits<double>::infinity()};
  return v[next() % 10];
}

static int32_t odd_count() {
  const int32_t v[] = {0, 1, 2, 4, 5, 8, 9, -3, 255, 256, 1024, 1025, 100000};
  return v[next() % 13];
}

static void mutate(pdr_card& c) {
  const int k = (int)(next() % 14);
  const int calo = (int)(next() % 2), s = (int)(next() % PDR_MAXSEG), j = (int)(next() % PDR_MAXEDGE);
  switch (k) {
    case 0: c.nseg[calo] = odd_count(); break;
    case 1: c.seg_eta_hi[calo][s] = odd_value(); break;
    case 2: c.seg_neta[calo][s] = odd_count(); break;
    case 3: c.seg_nphi[calo][s] = odd_count(); break;
    case 4: c.trk_npt = odd_count(); break;
    case 5: c.trk_eta_edges[j] = odd_value(); break;
    case 6: c.trk_eff[next() % 3][j][next() % PDR_MAXEDGE] = odd_value(); break;
    case 7: c.res_n[next() % 4] = odd_count(); break;
    case 8: c.res_abcd[next() % 4][j][next() % 4] = odd_value(); break;
    case 9: c.id_n = odd_count(); break;
    case 10: c.id_eff[next() % 3][j] = odd_value(); break;
    case 11: c.B = odd_value(); break;
    case 12: c.R = odd_value(); c.L = odd_value(); break;
    default: c.iso_dr = odd_value(); c.e_min[calo] = odd_value(); break;
  }
}

int main(int argc, char** argv) {
  if (argc != 2) return 2;
  FILE* f = std::fopen(argv[1], "rb");
  if (!f) return 2;
  std::vector<pdr_card> cards;
  pdr_card c;
  while (std::fread(&c, sizeof c, 1, f) == 1) cards.push_back(c);
  std::fclose(f);
  if (cards.empty()) return 2;
  auto dev = std::make_unique<pdr::DevCard>();
  std::vector<unsigned char> hot(PDR_HOT_MAX_BYTES);
  int accepted = 0, rejected = 0;
  for (const pdr_card& base : cards) {
    if (pdr::expand_card(&base, *dev) != PDR_OK) { std::fprintf(stderr, "a stock card was rejected\n"); return 1; }
    if (pdr::build_hot_card(*dev, hot.data(), hot.size()) == 0) { std::fprintf(stderr, "no card image\n"); return 1; }
    for (int trial = 0; trial < 3000; ++trial) {
      pdr_card m = base;
      const int n_mut = 1 + (int)(next() % 3);
      for (int k = 0; k < n_mut; ++k) mutate(m);
      if (pdr::expand_card(&m, *dev) == PDR_OK) {
        ++accepted;
        (void)pdr::build_hot_card(*dev, hot.data(), hot.size());
      } else {
        ++rejected;
      }
    }
  }
  std::printf("ok %d accepted, %d rejected\n", accepted, rejected);
  return 0;
}
