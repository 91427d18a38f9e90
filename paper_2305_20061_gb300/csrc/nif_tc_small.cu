// Tensor-core NIF of widths 64 and 32 (the narrower networks of the
// model-size study, Section 4.6); the kernel is in nif_tc.cuh.
#include "nif_tc.cuh"

namespace ptk {
namespace tcnif {

PT_NIF_TC_WIDTH(64)
PT_NIF_TC_WIDTH(32)

}  // namespace tcnif
}  // namespace ptk
