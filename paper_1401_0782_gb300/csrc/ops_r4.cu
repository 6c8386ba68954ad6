// Operator-kernel instantiations for the order-8 finite-difference stencil.
#include "ops_kernel.cuh"
RSN_INSTANTIATE_OPS(4)
