// Kernel instantiations and launch code for polynomial degree N = 1.
#include "ops_impl.cuh"
DG_DEFINE_N(1)
