// Explicit instantiations of the marching kernel's launcher, group 7 (see march_kernel.cuh).
#include "march_kernel.cuh"

HHG_MARCH_SHARD_7(HHG_MARCH_INSTANTIATE)
