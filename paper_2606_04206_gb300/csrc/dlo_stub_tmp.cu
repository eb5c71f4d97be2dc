#include "dlo_runtime.h"
extern "C" dlo_status dlo_step_plain(dlo_ctx* c, const float*, int, int) {
    if (!c) return DLO_ERR_INVALID_ARG;
    return set_err(c, DLO_ERR_STATE, "plain comparator not built");
}
