// Mixed-precision stage kernels for 4 LGL nodes per axis.
#include "dg_mixed.cuh"
DG_INSTANTIATE_MIXED(4)
