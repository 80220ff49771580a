// Kernel instantiations for N = 3 phases.
#include "ac_launch.cuh"
namespace ac {
const Ops *ops_n3() { return Launch<3>::table(); }
}  // namespace ac
