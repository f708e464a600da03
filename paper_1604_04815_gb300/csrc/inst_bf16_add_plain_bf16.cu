// Instantiations of the scan kernel for kind bf16_add_plain_bf16.
#include "kernel_inst.cuh"
namespace lscan {
using Kind_bf16_add_plain_bf16 = KFAddPlain<uint16_t, uint16_t>;
void register_bf16_add_plain_bf16() { fill_kind<Kind_bf16_add_plain_bf16>(KIND_BF16_ADD_PLAIN_BF16); }
}  // namespace lscan
