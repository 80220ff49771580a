// Kernel instantiations for N = 5 phases.
#include "ac_launch.cuh"
namespace ac {
const Ops *ops_n5() { return Launch<5>::table(); }
}  // namespace ac
