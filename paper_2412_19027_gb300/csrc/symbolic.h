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
  // forward solve: the same for the work vector w (one slot per front row)
  std::vector<int64_t> sv_lev_ptr, sv_tgt, sv_ptr, sv_src;
  std::vector<int32_t> rows_kkt;   // KKT index of every front row
};

void build_numeric_maps(const Symbolic& sy, const std::vector<int64_t>& kcol_ptr, const std::vector<int64_t>& krow,
                        NumericMaps& mp);

}  // namespace clr
