// Instantiations of the scan kernel for kind f32_add_f64.
#include "kernel_inst.cuh"
namespace lscan {
using Kind_f32_add_f64 = KFAddF64<float, float>;
void register_f32_add_f64() { fill_kind<Kind_f32_add_f64>(KIND_F32_ADD_F64); }
}  // namespace lscan
