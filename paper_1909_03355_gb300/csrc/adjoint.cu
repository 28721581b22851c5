// Reverse-time discrete adjoint (fedfem_forward_record / fedfem_adjoint).
#include "ctx.h"

using namespace fedfem;

extern "C" fedfem_status fedfem_forward_record(fedfem_ctx *c, int64_t, const int32_t *, int32_t, int32_t, int32_t,
                                               double *)
{
    return fail(c, FEDFEM_ERR_UNSUPPORTED, "adjoint not built yet");
}

extern "C" fedfem_status fedfem_adjoint(fedfem_ctx *c, const double *, double *, double *)
{
    return fail(c, FEDFEM_ERR_UNSUPPORTED, "adjoint not built yet");
}
