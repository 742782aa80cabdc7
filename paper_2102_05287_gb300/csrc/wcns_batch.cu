// Batched mode of the C ABI (placeholder until the batched kernels land).
#include "../../include/wcns.h"

extern "C" {
int wcns_batch_create(int, const int *, const double *, const double *, int, int, double, double, double,
                      wcns_batch **out) {
  if (out) *out = 0;
  return WCNS_E_UNSUPPORTED;
}
int wcns_batch_set_options(wcns_batch *, const wcns_options *) { return WCNS_E_UNSUPPORTED; }
int wcns_batch_advance(wcns_batch *, double *, int, double, double *) { return WCNS_E_UNSUPPORTED; }
int wcns_batch_get_stats(wcns_batch *, wcns_stats *) { return WCNS_E_UNSUPPORTED; }
long long wcns_batch_total_cells(const wcns_batch *) { return 0; }
long long wcns_batch_launch_count(const wcns_batch *) { return 0; }
void wcns_batch_destroy(wcns_batch *) {}
}
