// Instantiations of the scan kernel for kind i32_max.
#include "kernel_inst.cuh"
namespace lscan {
using Kind_i32_max = KI32Max;
void register_i32_max() { fill_kind<Kind_i32_max>(KIND_I32_MAX); }
}  // namespace lscan
