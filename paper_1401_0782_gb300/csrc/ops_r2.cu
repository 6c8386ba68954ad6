// Operator-kernel instantiations for the order-4 finite-difference stencil.
#include "ops_kernel.cuh"
RSN_INSTANTIATE_OPS(2)
