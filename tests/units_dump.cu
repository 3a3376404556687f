// Host-only dump of the column-walk plan the library's planner makes
// (column_chunk, column_segments, column_unit from csrc/common.cuh), for the
// CPU test that checks every unit against the lattice geometry.  Output, one
// line per (L, mixed, tp): "L mixed tp U K" followed by the HP*K units as four
// integers each.
#include <cstdio>

#include "common.cuh"

int main() {
  const int tps[] = {32, 64, 96, 128, 160, 256, 384, 512};
  for (int L = 2; L <= 26; L += 2) {
    for (int mixed = 0; mixed < 2; ++mixed) {
      for (int tp : tps) {
        const int U = mpk::column_chunk(4, L, mixed != 0);
        const int K = mpk::column_segments(L, U, tp);
        const int n = L * L / 2 * K;
        std::printf("%d %d %d %d %d", L, mixed, tp, U, K);
        for (int u = 0; u < n; ++u) {
          const int4 d = mpk::column_unit(L, K, u);
          std::printf(" %d %d %d %d", d.x, d.y, d.z, d.w);
        }
        std::printf("\n");
      }
    }
  }
  return 0;
}
