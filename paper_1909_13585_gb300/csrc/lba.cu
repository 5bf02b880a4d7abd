// Buckling analysis and sensitivities (placeholder until the eigensolver lands).
#include "handle.h"

namespace tobk {

int compute_buckling(tobk_handle* h, double* lambda, tobk_solve_info* info) {
  (void)lambda;
  (void)info;
  return fail(h, TOBK_E_STATE, "buckling analysis not available in this build");
}

int compute_sensitivities(tobk_handle* h, double* dlam, double* dJ, bool out_on_device, tobk_solve_info* info) {
  (void)dlam;
  (void)dJ;
  (void)out_on_device;
  (void)info;
  return fail(h, TOBK_E_STATE, "sensitivities not available in this build");
}

}  // namespace tobk
