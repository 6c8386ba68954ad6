// Operator-kernel instantiations for the order-12 finite-difference stencil.
#include "ops_kernel.cuh"
RSN_INSTANTIATE_OPS(6)
