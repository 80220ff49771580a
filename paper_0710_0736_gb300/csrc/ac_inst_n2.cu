// Kernel instantiations for N = 2 phases.
#include "ac_launch.cuh"
namespace ac {
const Ops *ops_n2() { return Launch<2>::table(); }
}  // namespace ac
