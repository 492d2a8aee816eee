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
// Lane s keeps the best unmatched r of its column (ties to the lowest r) and
// looks again only when that r is taken: taking any other r leaves the
// column's maximum and its lowest-r tie where they were.
template <int RT>
__device__ void greedy_match_warp(const unsigned long long *key, int R, int *perm) {
  const int lane = threadIdx.x & 31;
  unsigned used_r = 0u;
  bool done = lane >= R;   // column matched (or past the rank)
  unsigned long long best = 0ull;
  int br = -1;
  auto scan = [&]() {
    best = 0ull;
    br = -1;
    for (int r = 0; r < R; ++r) {
      if ((used_r >> r) & 1u) continue;
      const unsigned long long v = key[r * RT + lane];
      if (br < 0 || v > best) { best = v; br = r; }
    }
  };
  if (!done) scan();
  for (int round = 0; round < R; ++round) {
    // warp argmax over lanes: larger value wins, ties to the lower lane (s);
    // lanes with nothing left carry -1 and never win
    unsigned long long wv = done ? 0ull : best;
    int wr = done ? -1 : br, ws = lane;
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long ov = __shfl_xor_sync(0xffffffffu, wv, o);
      const int our = __shfl_xor_sync(0xffffffffu, wr, o);
      const int ous = __shfl_xor_sync(0xffffffffu, ws, o);
      const bool take = our >= 0 && (wr < 0 || ov > wv || (ov == wv && ous < ws));
      if (take) { wv = ov; wr = our; ws = ous; }
    }
    if (wr < 0) break;   // every lane holds the same winner after the butterfly
    if (lane == 0) perm[ws] = wr;
    used_r |= 1u << wr;
    if (lane == ws) done = true;
    if (!done && br == wr) scan();
  }
  __syncwarp();
}

}  // namespace octen
