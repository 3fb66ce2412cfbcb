// Mixed-precision stage kernels for 8 LGL nodes per axis.
#include "dg_mixed.cuh"
DG_INSTANTIATE_MIXED(8)
