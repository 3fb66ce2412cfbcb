// Mixed-precision stage kernels for 6 LGL nodes per axis.
#include "dg_mixed.cuh"
DG_INSTANTIATE_MIXED(6)
