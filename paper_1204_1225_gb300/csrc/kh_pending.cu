// Entry points whose kernels are not in this build yet: they validate nothing and return
// KH_ERR_UNSUPPORTED with a message, so callers fail loudly instead of silently.
#include "kh_plan.h"

extern "C" {

kh_status kirchhoff_batched_prepare(int, const kh_job*, void*)
{
    return kh::set_error(KH_ERR_UNSUPPORTED, "kirchhoff_batched_prepare: not built into this library yet");
}

kh_status kirchhoff_migrate_batched(int, const kh_job*, void*)
{
    return kh::set_error(KH_ERR_UNSUPPORTED, "kirchhoff_migrate_batched: not built into this library yet");
}

}  // extern "C"
