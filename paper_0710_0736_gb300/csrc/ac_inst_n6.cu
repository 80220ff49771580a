// Kernel instantiations for N = 6 phases.
#include "ac_launch.cuh"
namespace ac {
const Ops *ops_n6() { return Launch<6>::table(); }
}  // namespace ac
