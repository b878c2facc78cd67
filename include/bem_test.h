/*
 * bem_test.h -- test hooks of the library behind include/bem.h.  They are not
 * part of the method (the paper has no counterpart): they let a test drive
 * the library's failure paths from the host, without faulting a GPU.
 */
#ifndef BEM_TEST_H
#define BEM_TEST_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/*
 * bem_test_fail_alloc_after -- inject allocation failures.  After n more
 * successful device or pinned-host allocations by the library (every
 * cudaMalloc / cudaMallocHost it makes, on any thread), each further one
 * fails as if the runtime had returned cudaErrorMemoryAllocation, without
 * calling it, until the hook is reset with n < 0.  n = 0 fails the next
 * allocation.  The calls that allocate then return BEM_ERR_OOM and release
 * what they had allocated; a mesh they were given stays usable.  Always
 * returns BEM_OK.
 */
int bem_test_fail_alloc_after(int64_t n);

/* Number of device and pinned-host allocations the library has attempted in
 * this process (injected failures included). */
int64_t bem_test_alloc_count(void);

/* Where the library considers array p to live for a mesh on device dev:
 * 0 host memory (staged through the library's buffers), 1 memory the
 * kernels on dev use directly (dev's memory or managed memory), 2 another
 * GPU's memory (every entry point rejects it with BEM_ERR_INVALID). */
int32_t bem_test_ptr_location(const void* p, int32_t dev);

#ifdef __cplusplus
}
#endif

#endif /* BEM_TEST_H */
