// Instantiations of the scan kernel for kind f32_add_df.
#include "kernel_inst.cuh"
namespace lscan {
using Kind_f32_add_df = KFAddDF<float, float>;
void register_f32_add_df() { fill_kind<Kind_f32_add_df>(KIND_F32_ADD_DF); }
}  // namespace lscan
