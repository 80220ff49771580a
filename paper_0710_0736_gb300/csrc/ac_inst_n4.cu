// Kernel instantiations for N = 4 phases.
#include "ac_launch.cuh"
namespace ac {
const Ops *ops_n4() { return Launch<4>::table(); }
}  // namespace ac
