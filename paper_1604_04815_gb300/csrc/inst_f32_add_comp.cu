// Instantiations of the scan kernel for kind f32_add_comp.
#include "kernel_inst.cuh"
namespace lscan {
using Kind_f32_add_comp = KFAddComp<float, float>;
void register_f32_add_comp() { fill_kind<Kind_f32_add_comp>(KIND_F32_ADD_COMP); }
}  // namespace lscan
