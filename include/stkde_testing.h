/*
 * stkde_testing.h -- fault injection for tests of the library's error paths
 * (declared apart from stkde.h: production callers have no use for it).
 *
 * Each hook is armed on one context, applies once, and injects the failure on
 * the host side of the call or as a wait that nothing satisfies; none makes the
 * device fault.  What the tests check is that the failure is reported as the
 * documented status, that nothing leaks, and that the context computes
 * correctly afterwards.
 */
#ifndef STKDE_TESTING_H
#define STKDE_TESTING_H

#include "stkde.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    /* clears any armed fault of the context */
    STKDE_FAULT_NONE = 0,
    /* the arg-th device allocation the context makes from now on (workspace,
     * result buffer for host outputs, staging of host bandwidth arrays; arg >= 1)
     * fails as on a device out of memory: the call returns STKDE_ERR_OOM before
     * enqueueing anything and the buffer that was being grown is left empty */
    STKDE_FAULT_ALLOC = 1,
    /* the next tensor-form tile-kernel launch of the context: block 0 never
     * signals the arrival of its first staging page of stream 0 (and issues no
     * copy into it), and every wait of that launch gives up after arg
     * microseconds (1 <= arg <= 2,000,000).  The waits on that page then expire,
     * the block aborts (every role leaves its loop, copies and MMAs in flight
     * are drained, tensor memory is freed) and stkde_synchronize returns
     * STKDE_ERR_TIMEOUT; the grid is not valid.  Other blocks finish their tiles. */
    STKDE_FAULT_WITHHOLD_PAGE = 2
} stkde_fault;

/* Arms `fault` with argument `arg` on ctx.  Errors: INVALID_ARGUMENT (NULL ctx,
 * an unknown fault, arg out of range). */
STKDE_API stkde_status stkde_inject_fault(stkde_ctx* ctx, int fault, int64_t arg);

#ifdef __cplusplus
}
#endif

#endif /* STKDE_TESTING_H */
