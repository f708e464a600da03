// Instantiations of the scan kernel for kind i64_add.
#include "kernel_inst.cuh"
namespace lscan {
using Kind_i64_add = KI64Add;
void register_i64_add() { fill_kind<Kind_i64_add>(KIND_I64_ADD); }
}  // namespace lscan
