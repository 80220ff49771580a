// Kernel instantiations for N = 7 phases.
#include "ac_launch.cuh"
namespace ac {
const Ops *ops_n7() { return Launch<7>::table(); }
}  // namespace ac
