// Instantiations of the scan kernel for kind f32_add_plain.
#include "kernel_inst.cuh"
namespace lscan {
using Kind_f32_add_plain = KFAddPlain<float, float>;
void register_f32_add_plain() { fill_kind<Kind_f32_add_plain>(KIND_F32_ADD_PLAIN); }
}  // namespace lscan
