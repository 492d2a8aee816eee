// Greedy one-to-one matching of the factor match (Sec. "Factor match for
// identifiability"): repeatedly take the largest similarity among the columns
// not yet matched on either side, ties to the lowest reference column s and
// then the lowest replica column r.  Similarities are non-negative doubles,
// compared through their bit patterns (which order like the values) with
// integer instructions.
#pragma once

#include "octen_internal.cuh"

namespace octen {

// Warp 0 only (all 32 lanes): key[r * RT + s] = bits of sim(r, s) >= 0 for
// r, s < R <= 32.  Writes perm[s] = matched r for every s < R (shared memory).
template <int RT>
__device__ void greedy_match_warp(const unsigned long long *key, int R, int *perm) {
  const int lane = threadIdx.x & 31;
  unsigned used_r = 0u, used_s = 0u;
  for (int round = 0; round < R; ++round) {
    unsigned long long best = 0ull;
    int br = -1;
    if (lane < R && !((used_s >> lane) & 1u)) {
      for (int r = 0; r < R; ++r) {
        if ((used_r >> r) & 1u) continue;
        const unsigned long long v = key[r * RT + lane];
        if (br < 0 || v > best) { best = v; br = r; }
      }
    }
    // warp argmax over lanes: larger value wins, ties to the lower lane (s);
    // lanes with nothing left carry br = -1 and never win
    int bs = lane;
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int obr = __shfl_xor_sync(0xffffffffu, br, o);
      const int obs = __shfl_xor_sync(0xffffffffu, bs, o);
      const bool take = obr >= 0 && (br < 0 || ov > best || (ov == best && obs < bs));
      if (take) { best = ov; br = obr; bs = obs; }
    }
    if (br < 0) break;   // every lane holds the same winner after the butterfly
    if (lane == 0) perm[bs] = br;
    used_r |= 1u << br;
    used_s |= 1u << bs;
  }
  __syncwarp();
}

}  // namespace octen
