// Index maps of the numeric multifrontal LDL^T (built once at setup).
#pragma once

#include <cstdint>
#include <vector>

#include "internal.h"

namespace clr {

struct NumericMaps {
  std::vector<int64_t> kdest;      // kval entry -> pool position
  std::vector<int64_t> diag_pos;   // elimination position k -> pool position of (k, k)
  // factor extend-add: target pool positions of fronts at level l are
  // fa_tgt[fa_lev_ptr[l] .. fa_lev_ptr[l+1]); target t sums pool entries
  // fa_src[fa_ptr[t] .. fa_ptr[t+1]) (children's update matrices)
  std::vector<int64_t> fa_lev_ptr, fa_tgt, fa_ptr, fa_src;
  // extend-add of the large update blocks by relative indices (no per-entry map):
  // round k of level l adds the update block of the k-th such child of every
  // front of level l (at most one child per front per round, rounds in a fixed
  // order after the pull above, so every sum is taken in a fixed order).
  // Rounds of level l: px_round_ptr[px_lev_ptr[l] .. px_lev_ptr[l+1]] bound
  // ranges of px_child; rel[rel_off[J] + a] = row of the parent front that
  // receives update row a of child J.
  std::vector<int64_t> px_lev_ptr, px_round_ptr, px_child, rel_off;
  std::vector<int32_t> rel;
  // forward solve: the same for the work vector w (one slot per front row)
  std::vector<int64_t> sv_lev_ptr, sv_tgt, sv_ptr, sv_src;
  std::vector<int32_t> rows_kkt;   // KKT index of every front row
};

// direct = false builds every extend-add list by sorting pairs (the same lists).
void build_numeric_maps(const Symbolic& sy, const std::vector<int64_t>& kcol_ptr, const std::vector<int64_t>& krow,
                        NumericMaps& mp, bool direct = true);
// A hash (FNV-1a's step over whole entries) of the elimination order and every
// array of the maps.
uint64_t maps_digest(const Symbolic& sy, const NumericMaps& mp);

}  // namespace clr
