// Instantiations of the scan kernel for kind bf16_add_df_f32.
#include "kernel_inst.cuh"
namespace lscan {
using Kind_bf16_add_df_f32 = KFAddDF<uint16_t, float>;
void register_bf16_add_df_f32() { fill_kind<Kind_bf16_add_df_f32>(KIND_BF16_ADD_DF_F32); }
}  // namespace lscan
