// Kernel instantiations and launch code for polynomial degree N = 2.
#include "ops_impl.cuh"
DG_DEFINE_N(2)
