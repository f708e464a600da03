// Instantiations of the scan kernel for kind bf16_max.
#include "kernel_inst.cuh"
namespace lscan {
using Kind_bf16_max = KFMax<uint16_t>;
void register_bf16_max() { fill_kind<Kind_bf16_max>(KIND_BF16_MAX); }
}  // namespace lscan
