// Host-side check of the tile tables of the row-block-tiled Gram (gram_tiles): for R = 3
// and 4 row blocks, wide (BF16 / E4M3) and narrow (split BF16) tables must cover every
// block of the upper block triangle exactly once, read each segment's operands from the
// blocks the tile loads, and use at most the 512 tensor-memory columns of one CTA.
// Prints "ALL OK" and exits 0 when every check holds. Needs no GPU.
#include <algorithm>
#include <cstdio>
#include <set>
#include <utility>

#include "internal.h"

namespace pidk {
int gram_tiles(int R, bool wide, TileDesc* out);
size_t gram_tiled_smem_bytes(int prec, int slots, int stages);
}  // namespace pidk

using namespace pidk;

int main() {
  int bad = 0;
  for (int wide = 0; wide < 2; ++wide) {
    for (int R = 3; R <= 4; ++R) {
      TileDesc t[kMaxTiles];
      const int n = gram_tiles(R, wide != 0, t);
      if (n < 1 || n > kMaxTiles) { std::printf("R=%d wide=%d: %d tiles\n", R, wide, n); ++bad; continue; }
      std::set<std::pair<int, int>> seen;
      int slots = 0;
      for (int k = 0; k < n; ++k) {
        const TileDesc& d = t[k];
        slots = std::max(slots, d.nlb + (d.xa >= 0 ? 1 : 0));
        int cols = 0;
        for (int s = 0; s < d.nseg; ++s) {
          const bool a_in = (d.ra[s] >= d.lb0 && d.ra[s] < d.lb0 + d.nlb) || d.ra[s] == d.xa;
          const bool b_in = d.cb[s] >= d.lb0 && d.cb[s] + d.nb[s] <= d.lb0 + d.nlb;
          if (!a_in || !b_in || d.col[s] != cols) {
            std::printf("R=%d wide=%d tile %d segment %d: operands or columns out of place\n", R, wide, k, s);
            ++bad;
          }
          cols += 128 * d.nb[s];
          for (int b = d.cb[s]; b < d.cb[s] + d.nb[s]; ++b) {
            if (b < d.ra[s] || b >= R || !seen.insert({d.ra[s], b}).second) {
              std::printf("R=%d wide=%d: block (%d, %d) below the diagonal, outside or twice\n", R, wide, d.ra[s], b);
              ++bad;
            }
          }
        }
        if (cols > 512) { std::printf("R=%d wide=%d tile %d: %d columns\n", R, wide, k, cols); ++bad; }
      }
      if (static_cast<int>(seen.size()) != R * (R + 1) / 2) {
        std::printf("R=%d wide=%d: %zu of %d blocks covered\n", R, wide, seen.size(), R * (R + 1) / 2);
        ++bad;
      }
      // the ring must hold at least two stages in the 227 KB of shared memory of a CTA, for
      // every precision that uses the table (split BF16 takes the wide one for R = 3 only)
      for (int prec = 1; prec <= 3; ++prec) {
        const bool uses = wide ? (prec != 2 || R == 3) : (prec == 2 && R != 3);
        if (uses && gram_tiled_smem_bytes(prec, slots, 2) > 232448) {
          std::printf("R=%d wide=%d prec=%d: two stages of %d slots do not fit\n", R, wide, prec, slots);
          ++bad;
        }
      }
    }
  }
  std::printf(bad ? "FAILED %d\n" : "ALL OK\n", bad);
  return bad != 0;
}
