// Mixed-precision contractions: not built yet in this file revision.
#include "gw_internal.h"
#include "gw_mixed.h"

namespace gwi {

struct MixedState {
  MixedDims d;
};

int mixed_create(MixedState** out, const MixedDims& d, cudaStream_t, size_t*) {
  *out = nullptr;
  (void)d;
  return fail(GW_ENOTIMPL, "mixed precision is not available in this build");
}
void mixed_destroy(MixedState* s) { delete s; }
int mixed_set_coulomb(MixedState*, const double2*, const long long*) { return fail(GW_ENOTIMPL, "mixed"); }
int mixed_polarization(MixedState*, const double2*, double2*, double) { return fail(GW_ENOTIMPL, "mixed"); }
int mixed_self_energy(MixedState*, const double2*, const double2*, double2*) { return fail(GW_ENOTIMPL, "mixed"); }

}  // namespace gwi
