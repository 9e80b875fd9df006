// FP64 instantiation of the MRA kernels (r_hat padded to 16 or 32).
#include "mra_launch.cuh"
namespace mra {
MRA_INSTANTIATE(double, 16)
MRA_INSTANTIATE(double, 32)
MRA_INSTANTIATE_DOWN(16)
MRA_INSTANTIATE_DOWN(32)
} // namespace mra
