// FP64 stage kernels for 7 LGL nodes per axis.
#include "dg_stage_fp64.cuh"
DG_INSTANTIATE_STAGE(7)
