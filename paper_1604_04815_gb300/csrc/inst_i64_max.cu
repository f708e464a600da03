// Instantiations of the scan kernel for kind i64_max.
#include "kernel_inst.cuh"
namespace lscan {
using Kind_i64_max = KI64Max;
void register_i64_max() { fill_kind<Kind_i64_max>(KIND_I64_MAX); }
}  // namespace lscan
