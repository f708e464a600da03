// Instantiations of the scan kernel for kind i32_add.
#include "kernel_inst.cuh"
namespace lscan {
using Kind_i32_add = KI32Add;
void register_i32_add() { fill_kind<Kind_i32_add>(KIND_I32_ADD); }
}  // namespace lscan
