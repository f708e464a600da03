// Instantiations of the stream-compaction kernels (2-, 4- and 8-byte values).
#include "kernel_inst.cuh"
namespace lscan {
void register_select() {
    fill_select<KSelect<uint16_t>>(KIND_SEL16);
    fill_select<KSelect<uint32_t>>(KIND_SEL32);
    fill_select<KSelect<uint64_t>>(KIND_SEL64);
}
}  // namespace lscan
