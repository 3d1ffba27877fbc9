/*
 * lbm_testing.h -- test hooks of liblbm_gb300: host-side fault injection for the tests of
 * the library's error paths. None of them makes the GPU fault; each fakes the failure of
 * a call on the host or plants the record a failed device-side check would leave.
 * The paper has no counterpart (its kernels have no error handling to test).
 *
 * Ownership and errors follow include/lbm.h. These hooks change process-wide state
 * (the allocation counter and the injected failure); they are not thread-safe against
 * concurrent use of the library.
 */
#ifndef LBM_GB300_TESTING_H
#define LBM_GB300_TESTING_H

#include <stdint.h>

#include "lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Device buffers the library holds now (every context, every call in progress). A
 * context that failed to build, and every call that failed, must leave it unchanged. */
int64_t lbm_testing_live_allocations(void);

/* Make the k-th device allocation from now on (k = 0: the next one) fail the way
 * cudaMalloc fails when device memory runs out; the call that made it returns
 * LBM_ENOMEM after releasing what it had allocated. k < 0 cancels the injection. One
 * failure per call of this hook. */
void lbm_testing_fail_allocation(int64_t k);

/* 1 if this library was built with LBM_CHECKED: the step kernel then tests every work-
 * group header, node tile and gather source against the context's arrays before it uses
 * them; a failed test skips the access and records (code << 56) | value in the context's
 * error word, and lbm_step / lbm_step_kernel return LBM_EINTERNAL (sticky). Codes:
 * 1 header, 2 node tile, 3 gather source outside the population copy. */
int lbm_testing_checked_build(void);

/* Checked build only: store `word` in the context's error word, as a failed check would,
 * so that the host side of the mechanism can be tested without an out-of-range index.
 * LBM_EUNSUPPORTED in the normal build. */
lbm_status lbm_testing_plant_check(lbm_ctx* ctx, uint64_t word);

#ifdef __cplusplus
}
#endif
#endif /* LBM_GB300_TESTING_H */
