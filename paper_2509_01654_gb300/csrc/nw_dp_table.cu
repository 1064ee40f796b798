// Maps a length LB to its alignment kernel across the instantiation units.
#include "nw_launch.h"

namespace nw {
const void* dp_kernel_range_0(int LB, int epi, bool tab);
const void* dp_kernel_range_11(int LB, int epi, bool tab);
const void* dp_kernel_range_21(int LB, int epi, bool tab);
const void* dp_kernel_range_31(int LB, int epi, bool tab);

const void* dp_kernel(int LB, int epi, bool tab) {
  if (LB < 0 || LB > kMaxLen) return nullptr;
  if (LB <= 10) return dp_kernel_range_0(LB, epi, tab);
  if (LB <= 20) return dp_kernel_range_11(LB, epi, tab);
  if (LB <= 30) return dp_kernel_range_21(LB, epi, tab);
  return dp_kernel_range_31(LB, epi, tab);
}
}  // namespace nw
