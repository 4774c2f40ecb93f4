// batch.cu -- many independent 2D problems in one persistent launch.
#include "acs_host.h"

extern "C" {
ACS_API int acs_batch_create(int, const int64_t*, const double*, const double*, const double*, const int*, int,
                             acs_batch**) { return ACS_E_UNSUPPORTED; }
ACS_API size_t acs_batch_numel(const acs_batch*) { return 0; }
ACS_API int acs_batch_offsets(const acs_batch*, int64_t*) { return ACS_E_UNSUPPORTED; }
ACS_API size_t acs_batch_work_bytes(const acs_batch*) { return 0; }
ACS_API int acs_batch_bind(acs_batch*, void*, void*, size_t, void*) { return ACS_E_UNSUPPORTED; }
ACS_API int acs_batch_step(acs_batch*, int64_t) { return ACS_E_UNSUPPORTED; }
ACS_API int acs_batch_observe(acs_batch*, double*, double*) { return ACS_E_UNSUPPORTED; }
ACS_API void acs_batch_destroy(acs_batch*) {}
}
