// Explicit instantiations of the marching kernel's launcher, group 6 (see march_kernel.cuh).
#include "march_kernel.cuh"

HHG_MARCH_SHARD_6(HHG_MARCH_INSTANTIATE)
