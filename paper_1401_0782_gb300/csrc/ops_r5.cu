// Operator-kernel instantiations for the order-10 finite-difference stencil.
#include "ops_kernel.cuh"
RSN_INSTANTIATE_OPS(5)
