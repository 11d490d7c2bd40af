/*
 * rb_testing.h -- test hooks of the greedy reduced-basis library.  Not part
 * of the method's interface (include/rb.h); the tests call these to exercise
 * failure handling without faulting, trapping or hanging a GPU.  The paper
 * has no counterpart.
 */
#ifndef RB_GB300_TESTING_H
#define RB_GB300_TESTING_H

#include "rb.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Self-test of the bounded device-side wait every tensor-core kernel uses:
 * one thread waits on an mbarrier that nothing arrives on (arrive = 0) for at
 * most `cycles` SM clock cycles, then records a time-out and the kernel
 * returns normally.  Returns RB_ETIMEOUT when the wait ran out (expected for
 * arrive = 0), RB_OK when it completed (arrive = 1), RB_EINVAL for cycles < 1
 * or a null ctx, RB_ECUDA when a CUDA call fails. */
rb_status rb_debug_wait_selftest(rb_ctx *ctx, long long cycles, int arrive);

#ifdef __cplusplus
}
#endif
#endif /* RB_GB300_TESTING_H */
