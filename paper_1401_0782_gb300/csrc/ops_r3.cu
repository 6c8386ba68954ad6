// Operator-kernel instantiations for the order-6 finite-difference stencil.
#include "ops_kernel.cuh"
RSN_INSTANTIATE_OPS(3)
