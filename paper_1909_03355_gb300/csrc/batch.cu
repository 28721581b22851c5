// Batched scenarios (fedfem_batch_*).
#include "ctx.h"

struct fedfem_batch {
    std::string err;
};

extern "C" fedfem_status fedfem_batch_create(const fedfem_scenario *, int32_t, const fedfem_options *, fedfem_batch **out)
{
    if (out) *out = nullptr;
    return FEDFEM_ERR_UNSUPPORTED;
}
extern "C" fedfem_status fedfem_batch_run(fedfem_batch *) { return FEDFEM_ERR_UNSUPPORTED; }
extern "C" fedfem_status fedfem_batch_times(fedfem_batch *, double *, double *, double *) { return FEDFEM_ERR_UNSUPPORTED; }
extern "C" fedfem_status fedfem_batch_get_T(fedfem_batch *, int32_t, double *) { return FEDFEM_ERR_UNSUPPORTED; }
extern "C" const char *fedfem_batch_error_string(fedfem_batch *b) { return b ? b->err.c_str() : "NULL batch"; }
extern "C" void fedfem_batch_destroy(fedfem_batch *b) { delete b; }
