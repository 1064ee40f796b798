// Alignment kernels for the longer word length LB in [0, 10].
#define NW_LB_LO 0
#define NW_LB_HI 10
#include "nw_dp_inst.inc"
