// Instantiations of the scan kernel for kind bf16_add_df_bf16.
#include "kernel_inst.cuh"
namespace lscan {
using Kind_bf16_add_df_bf16 = KFAddDF<uint16_t, uint16_t>;
void register_bf16_add_df_bf16() { fill_kind<Kind_bf16_add_df_bf16>(KIND_BF16_ADD_DF_BF16); }
}  // namespace lscan
