// Alignment kernels for the longer word length LB in [21, 30].
#define NW_LB_LO 21
#define NW_LB_HI 30
#include "nw_dp_inst.inc"
