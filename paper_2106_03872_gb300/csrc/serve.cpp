// Serving entry points (placeholder until the scheduler is built).
#include "common.h"

extern "C" {
ks_status ks_serve_create(size_t, ks_server* out) {
  if (out) *out = nullptr;
  ks::set_last_error("serving scheduler not built yet");
  return KS_ERR_STATE;
}
ks_status ks_serve_destroy(ks_server) { return KS_OK; }
ks_status ks_serve_submit(ks_server, const ks_cell_desc*, const double*, int, int, double, uint64_t*) {
  ks::set_last_error("serving scheduler not built yet");
  return KS_ERR_STATE;
}
ks_status ks_serve_poll(ks_server, uint64_t, int, double*, double*, double*) {
  ks::set_last_error("serving scheduler not built yet");
  return KS_ERR_STATE;
}
ks_status ks_serve_result_info(ks_server, uint64_t, int*, int*, int*) {
  ks::set_last_error("serving scheduler not built yet");
  return KS_ERR_STATE;
}
}
