// Kernel instantiations for N = 8 phases.
#include "ac_launch.cuh"
namespace ac {
const Ops *ops_n8() { return Launch<8>::table(); }
}  // namespace ac
