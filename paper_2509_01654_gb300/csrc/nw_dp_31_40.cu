// Alignment kernels for the longer word length LB in [31, 40].
#define NW_LB_LO 31
#define NW_LB_HI 40
#include "nw_dp_inst.inc"
