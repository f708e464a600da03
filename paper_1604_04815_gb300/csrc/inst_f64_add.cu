// Instantiations of the scan kernel for kind f64_add.
#include "kernel_inst.cuh"
namespace lscan {
using Kind_f64_add = KF64Add;
void register_f64_add() { fill_kind<Kind_f64_add>(KIND_F64_ADD); }
}  // namespace lscan
