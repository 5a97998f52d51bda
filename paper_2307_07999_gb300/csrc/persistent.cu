// Persistent batched kernel (filled in below).
#include "batch.h"
glasma_status batch_run_persistent(glasma_batch* b) {
    (void)b;
    glasma_set_error("persistent mode not built");
    return GLASMA_ERR_INVALID;
}
void batch_free_persistent(glasma_batch* b) { (void)b; }
