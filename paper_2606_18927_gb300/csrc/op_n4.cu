// Kernel instantiations and launch code for polynomial degree N = 4.
#include "ops_impl.cuh"
DG_DEFINE_N(4)
