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

/*
 * bem_test_rule_records -- the far-field kernels' node records of rule r
 * (0..4, the 4-, 7-, 12-, 19|17- and 33-point rule) of element type `type`
 * (BEM_TRIANGLE or BEM_RECTANGLE), as built on the host for the mixed
 * (precision 1, FP32 values) or the FP64 (precision 0) path: the centre node
 * first (if the rule has one), then one record per pair of nodes o, -o of
 * equal weight (rectangles) or one per node (triangles).  Writes one row
 * (alpha, beta, w, multiplicity) per record to out (at most 33 rows, host
 * memory), the multiplicity being 2 for a pair and 1 otherwise, and *shape =
 * centre records | other records << 1.  Returns the number of records, or
 * BEM_ERR_INVALID for bad arguments.  Needs no GPU.
 */
int32_t bem_test_rule_records(int32_t type, int32_t r, int32_t precision, double* out /* 33 x 4 */, int32_t* shape);

#ifdef __cplusplus
}
#endif

#endif /* BEM_TEST_H */
