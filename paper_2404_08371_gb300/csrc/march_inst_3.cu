// Explicit instantiations of the marching kernel's launcher, group 3 (see march_kernel.cuh).
#include "march_kernel.cuh"

HHG_MARCH_SHARD_3(HHG_MARCH_INSTANTIATE)
