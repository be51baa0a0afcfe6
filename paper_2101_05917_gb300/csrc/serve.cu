// Continuous-batching server for rollout-plus-gradient requests.
#include "pd_internal.cuh"

extern "C" {

pd_status pd_serve_create(int32_t, size_t, int32_t, pd_server* out) {
  if (out) *out = nullptr;
  pd::set_error("pd_serve_create: serving is not built yet");
  return PD_ERR_INVALID_ARG;
}
pd_status pd_serve_submit(pd_server, const pd_request*, uint64_t*) {
  pd::set_error("pd_serve_submit: serving is not built yet");
  return PD_ERR_INVALID_ARG;
}
pd_status pd_serve_poll(pd_server, uint64_t, pd_result*) {
  pd::set_error("pd_serve_poll: serving is not built yet");
  return PD_ERR_INVALID_ARG;
}
pd_status pd_serve_drain(pd_server) { return PD_ERR_INVALID_ARG; }
void pd_serve_destroy(pd_server) {}

}  // extern "C"
