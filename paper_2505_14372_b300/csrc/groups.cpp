// Grouping of scan positions (arXiv 2505.14372 §2.2): per iteration, the
// positions are split into groups that are either sparse (random) or compact
// (spatially contiguous), and the order of the groups is shuffled.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <numeric>
#include <vector>

#include "errors.h"
#include "ptycho.h"

namespace {

// SplitMix64 (Steele, Lea, Flood 2014): a counter-based 64-bit generator.
struct SplitMix64 {
  uint64_t s;
  uint64_t next() {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  // uniform integer in [0, n) by rejection (no modulo bias)
  uint64_t below(uint64_t n) {
    const uint64_t lim = UINT64_MAX - UINT64_MAX % n;
    uint64_t x;
    do x = next(); while (x >= lim);
    return x % n;
  }
};

template <class T>
void shuffle(std::vector<T>& v, SplitMix64& r) {
  for (size_t i = v.size(); i > 1; --i) std::swap(v[i - 1], v[r.below(i)]);
}

// Interleave the bits of two 32-bit cell indices (Morton / Z order).
uint64_t morton(uint32_t y, uint32_t x) {
  auto spread = [](uint64_t v) {
    v &= 0xffffffffull;
    v = (v | (v << 16)) & 0x0000ffff0000ffffull;
    v = (v | (v << 8)) & 0x00ff00ff00ff00ffull;
    v = (v | (v << 4)) & 0x0f0f0f0f0f0f0f0full;
    v = (v | (v << 2)) & 0x3333333333333333ull;
    v = (v | (v << 1)) & 0x5555555555555555ull;
    return v;
  };
  return (spread(y) << 1) | spread(x);
}

}  // namespace

extern "C" int ptycho_make_groups(int32_t P, int32_t B, uint64_t seed, int64_t iteration, int32_t mode,
                                  const float* pos_host, int32_t* out_idx) {
  if (P < 0 || B < 1 || !out_idx || (mode != 0 && mode != 1)) return perr(PTYCHO_EINVAL, "bad grouping arguments");
  if (mode == 1 && P > 0 && !pos_host) return perr(PTYCHO_EINVAL, "compact grouping needs positions");
  SplitMix64 r{seed ^ (0xD1B54A32D192ED03ull * (uint64_t)(iteration + 1))};
  r.next();
  std::vector<int32_t> v(P);
  std::iota(v.begin(), v.end(), 0);
  if (mode == 0) {
    shuffle(v, r);
  } else {
    float y0 = 0, x0 = 0;
    if (P > 0) {
      y0 = pos_host[0];
      x0 = pos_host[1];
      for (int i = 1; i < P; ++i) {
        y0 = std::min(y0, pos_host[2 * i]);
        x0 = std::min(x0, pos_host[2 * i + 1]);
      }
    }
    std::vector<uint64_t> key(P);
    for (int i = 0; i < P; ++i)
      key[i] = morton((uint32_t)std::lround(pos_host[2 * i] - y0), (uint32_t)std::lround(pos_host[2 * i + 1] - x0));
    std::stable_sort(v.begin(), v.end(), [&](int a, int b) { return key[a] < key[b]; });
    // rotate by a random offset so group boundaries move between iterations
    if (P > 0) std::rotate(v.begin(), v.begin() + (long)r.below((uint64_t)P), v.end());
    const int ng = (P + B - 1) / B;
    std::vector<int> order(ng);
    std::iota(order.begin(), order.end(), 0);
    shuffle(order, r);
    std::vector<int32_t> out;
    out.reserve(P);
    for (int g : order)
      for (int i = g * B; i < std::min(P, (g + 1) * B); ++i) out.push_back(v[i]);
    v.swap(out);
  }
  std::copy(v.begin(), v.end(), out_idx);
  return PTYCHO_OK;
}
