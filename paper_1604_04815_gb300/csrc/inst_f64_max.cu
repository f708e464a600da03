// Instantiations of the scan kernel for kind f64_max.
#include "kernel_inst.cuh"
namespace lscan {
using Kind_f64_max = KF64Max;
void register_f64_max() { fill_kind<Kind_f64_max>(KIND_F64_MAX); }
}  // namespace lscan
