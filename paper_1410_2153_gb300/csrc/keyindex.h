// Position lookup in a sorted array of 64-bit keys (lattice or box Morton
// keys) through a table of bucket starts over the top key bits, used by the
// host setup for its many membership tests.
#pragma once

#include <algorithm>
#include <cstdint>
#include <vector>

namespace asmg {

// A short binary search inside one bucket instead of one over the whole
// array: the same positions as std::lower_bound.
struct KeyIndex {
  const std::vector<uint64_t>* keys = nullptr;
  int shift = 64;
  std::vector<int64_t> start;  // first position of bucket b; start[nb] = size
  void build(const std::vector<uint64_t>& k, int bits) {
    keys = &k;
    uint64_t top = k.empty() ? 0 : k.back();
    int hb = 0;
    while (hb < 64 && (top >> hb)) ++hb;
    shift = std::max(0, hb - bits);
    const int64_t nb = (int64_t)(top >> shift) + 1;
    start.assign(nb + 1, (int64_t)k.size());
    for (int64_t i = (int64_t)k.size() - 1; i >= 0; --i) start[k[i] >> shift] = i;
    for (int64_t b = nb - 1; b >= 0; --b) start[b] = std::min(start[b], start[b + 1]);
  }
  int32_t find(uint64_t x) const {
    const uint64_t b = x >> shift;
    if (b + 1 >= start.size()) return -1;
    auto lo = keys->begin() + start[b], hi = keys->begin() + start[b + 1];
    auto it = std::lower_bound(lo, hi, x);
    return (it != hi && *it == x) ? (int32_t)(it - keys->begin()) : -1;
  }
};

}  // namespace asmg
