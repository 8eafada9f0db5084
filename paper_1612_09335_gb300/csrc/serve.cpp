// Serving loop (continuous batching of independent solves).
#include "../../include/cweno.h"
#include "api_internal.h"

extern "C" {
int serve_create(size_t, int, int, cweno_server** out) {
  if (out) *out = nullptr;
  return cw::fail(CWENO_EINVAL, "serving is not built yet");
}
int serve_submit(cweno_server*, const cweno_request*, uint64_t*) { return cw::fail(CWENO_EINVAL, "no server"); }
int serve_poll(cweno_server*, uint64_t, int*, double*, double*) { return cw::fail(CWENO_EINVAL, "no server"); }
int serve_drain(cweno_server*, double) { return cw::fail(CWENO_EINVAL, "no server"); }
int serve_stats(cweno_server*, uint64_t*, uint64_t*, uint64_t*, uint64_t*, double*) {
  return cw::fail(CWENO_EINVAL, "no server");
}
void serve_destroy(cweno_server*) {}
}
