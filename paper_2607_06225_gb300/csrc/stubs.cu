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

filtr_status filtr_serve_create(filtr_ctx *, size_t, uint32_t, filtr_server **out) {
  if (out) *out = nullptr;
  set_error("serving is not available in this build");
  return FILTR_ERR_UNSUPPORTED;
}
filtr_status filtr_serve_submit(filtr_server *, const filtr_params *, const uint8_t *, uint32_t,
                                const uint8_t *, uint32_t, uint64_t *) {
  return FILTR_ERR_UNSUPPORTED;
}
filtr_status filtr_serve_poll(filtr_server *, uint64_t, filtr_result *, uint32_t *, uint64_t,
                              uint64_t *) {
  return FILTR_ERR_UNSUPPORTED;
}
filtr_status filtr_serve_wait(filtr_server *, uint64_t, int64_t, filtr_result *, uint32_t *,
                              uint64_t, uint64_t *) {
  return FILTR_ERR_UNSUPPORTED;
}
filtr_status filtr_serve_destroy(filtr_server *) { return FILTR_OK; }

}
