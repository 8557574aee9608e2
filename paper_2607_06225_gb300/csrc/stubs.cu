// stubs.cu -- entry points whose implementation lands in later files.
#include "filtr_ctx.h"

using namespace filtr;

extern "C" {

filtr_status filtr_align_long(filtr_ctx *, const filtr_params *, const uint8_t *, uint32_t,
                              const uint8_t *, uint32_t, filtr_result *, uint32_t *, uint64_t,
                              void *) {
  set_error("filtr_align_long is not available in this build");
  return FILTR_ERR_UNSUPPORTED;
}

}
