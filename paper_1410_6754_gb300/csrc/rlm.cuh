// Arguments of one RLM-sort level (Section 5): multisequence selection over the
// tiles of every part, then delivery of the pieces to the new parts.
#pragma once

#include "ams_internal.cuh"

namespace ams {

struct RlmArgs {
  const void* src;          // tiles of the current level (ordered keys)
  void* dst;                // delivery target (other buffer)
  const uint64_t* vsrc;     // payloads (pairs) or null
  uint64_t* vdst;
  const uint32_t* part_lo;  // nparts + 1 part boundaries of the current level
  uint32_t nparts;
  uint32_t r;               // new parts per part
  uint32_t run;             // tile size
  uint32_t max_tiles;       // largest tile count of a part (cut-table row stride)
  uint32_t* cuts;           // [nparts][r + 1][max_tiles] cut positions inside the tiles
  uint32_t* offs;           // [nparts][r][max_tiles] where each piece starts in its new part
  uint64_t seed;
  int level;
  uint32_t* status;
};

}  // namespace ams
