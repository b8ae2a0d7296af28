// Explicit instantiations of the marching kernel's launcher, group 0 (see march_kernel.cuh).
#include "march_kernel.cuh"

HHG_MARCH_SHARD_0(HHG_MARCH_INSTANTIATE)
