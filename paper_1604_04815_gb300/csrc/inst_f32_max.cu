// Instantiations of the scan kernel for kind f32_max.
#include "kernel_inst.cuh"
namespace lscan {
using Kind_f32_max = KFMax<float>;
void register_f32_max() { fill_kind<Kind_f32_max>(KIND_F32_MAX); }
}  // namespace lscan
