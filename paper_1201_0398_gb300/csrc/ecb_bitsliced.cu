// Bitsliced AES kernel (placeholder until the Boolean-circuit kernel lands).
#include "gbaes_internal.h"

namespace gbaes {

int launch_bitsliced(const EcbArgs&, int, Mode, int, cudaStream_t) {
    return fail(AES_ERR_ARG, "the bitsliced kernel is not built yet");
}

}  // namespace gbaes
