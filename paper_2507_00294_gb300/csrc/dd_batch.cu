// dd_batch.cu -- many scans in one launch (placeholder until the persistent kernel lands).
#include "dd_internal.h"

extern "C" dd_status dd_field_batch(const dd_scan *const *scans, int32_t n_scans, const int64_t *pt_offsets,
                                    const double *pts_xy_m, const double *times_s, dd_precision prec,
                                    double *out, void *cuda_stream) {
    (void)scans; (void)n_scans; (void)pt_offsets; (void)pts_xy_m; (void)times_s; (void)prec; (void)out;
    (void)cuda_stream;
    dd::clear_error();
    return dd::fail(DD_ENOTSUP, "dd_field_batch: not built yet");
}
