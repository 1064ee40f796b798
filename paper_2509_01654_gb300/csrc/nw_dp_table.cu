// Maps a length LB to its alignment kernel across the instantiation units.
#include "nw_launch.h"

namespace nw {
const void* dp_kernel_range_0(int LB, int epi);
const void* dp_kernel_range_11(int LB, int epi);
const void* dp_kernel_range_21(int LB, int epi);
const void* dp_kernel_range_31(int LB, int epi);

const void* dp_kernel(int LB, int epi) {
  if (LB < 0 || LB > kMaxLen) return nullptr;
  if (LB <= 10) return dp_kernel_range_0(LB, epi);
  if (LB <= 20) return dp_kernel_range_11(LB, epi);
  if (LB <= 30) return dp_kernel_range_21(LB, epi);
  return dp_kernel_range_31(LB, epi);
}
}  // namespace nw
