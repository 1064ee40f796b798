// Alignment kernels for the longer word length LB in [11, 20].
#define NW_LB_LO 11
#define NW_LB_HI 20
#include "nw_dp_inst.inc"
