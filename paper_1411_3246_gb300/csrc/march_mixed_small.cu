// Mixed form of the xi-march in tiles of 128 and 256 threads (several CTAs per SM), for
// simulations with few nodes and rings.
#include "march_tiles.cuh"

namespace wake {

bool march_tile_mixed_small(int nt, int ppt, TileFns *out) {
  if (nt == 128) {
    switch (ppt) {
      case 1: *out = tile_fns<PolMixed, 128, 1>(); return true;
      case 2: *out = tile_fns<PolMixed, 128, 2>(); return true;
      case 4: *out = tile_fns<PolMixed, 128, 4>(); return true;
      case 8: *out = tile_fns<PolMixed, 128, 8>(); return true;
      default: return false;
    }
  }
  if (nt == 256) {
    switch (ppt) {
      case 1: *out = tile_fns<PolMixed, 256, 1>(); return true;
      case 2: *out = tile_fns<PolMixed, 256, 2>(); return true;
      case 4: *out = tile_fns<PolMixed, 256, 4>(); return true;
      case 8: *out = tile_fns<PolMixed, 256, 8>(); return true;
      default: return false;
    }
  }
  return false;
}

}  // namespace wake
