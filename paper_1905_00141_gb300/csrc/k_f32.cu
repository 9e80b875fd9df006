// Mixed-precision instantiation: FP32 storage and products, FP64 factors,
// log-determinants and quadratic forms (r_hat padded to 16 or 32).
#include "mra_launch.cuh"
namespace mra {
MRA_INSTANTIATE(float, 16)
MRA_INSTANTIATE(float, 32)
} // namespace mra
