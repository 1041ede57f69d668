// Continuous-batching request server (energy + dE/dtheta solves).
#include <cuda_runtime.h>

#include "internal.h"

struct gocp_server {
  int placeholder;
};

using namespace gocp;

extern "C" {

int gocp_server_create(size_t, int, int, gocp_server** out) {
  if (out) *out = nullptr;
  return fail(GOCP_EINVAL, "server not available in this build");
}
void gocp_server_destroy(gocp_server*) {}
int gocp_submit(gocp_server*, const gocp_problem*, const int32_t*, const double*, int, uint64_t*) {
  return fail(GOCP_EINVAL, "server not available in this build");
}
int gocp_poll(gocp_server*, uint64_t, double*, double*, int64_t) {
  return fail(GOCP_EINVAL, "server not available in this build");
}
int gocp_cancel(gocp_server*, uint64_t) { return fail(GOCP_EINVAL, "server not available in this build"); }
int gocp_server_get_stats(gocp_server*, gocp_server_stats*) {
  return fail(GOCP_EINVAL, "server not available in this build");
}

}  // extern "C"
