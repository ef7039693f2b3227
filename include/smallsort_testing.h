/*
 * smallsort_testing.h -- test hook of libsmallsort.so.  Not for production
 * use.  (Library addition: the paper has no counterpart.)
 *
 * The failure paths of the kernels are exercised from the host: a flag makes
 * a kernel arm its copy-completion barrier without issuing the copy, so that
 * kernel's own bounded wait (sn_set_wait_limit) runs out, it records
 * SN_ETIMEOUT in the status word and returns.  Nothing faults and nothing
 * waits forever; the device stays usable.  The data of a call that ran with
 * a flag set is left unsorted or partly sorted.
 */
#ifndef SMALLSORT_TESTING_H
#define SMALLSORT_TESTING_H

#ifdef __cplusplus
extern "C" {
#endif

#define SN_TEST_SKIP_FIXED_COPY 1u /* fixed-size kernel (sn_sort_fixed*)                    */
#define SN_TEST_SKIP_TILE_COPY 2u  /* network tile kernel of the segmented calls (<= 32 items) */
#define SN_TEST_SKIP_RSS_COPY 4u   /* Register Sample Sort kernel (segments of 33..256)       */

/*
 * Sets the test flags of the current device (0 clears them; other bits:
 * SN_EINVAL).  Synchronous; call it while no library work runs on the device.
 */
int sn_test_set_flags(unsigned flags);

#ifdef __cplusplus
}
#endif

#endif /* SMALLSORT_TESTING_H */
