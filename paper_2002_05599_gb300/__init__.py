"""GB300-native batched small-set sorting.

Implements the hot path of Bingmann, Marianczuk, Sanders, "Engineering Faster
Sorters for Small Sets of Items" on one sm_103a GPU: branch-free sorting
networks for n <= 16 (Sec. 2), a 32-lane warp network for 17..32 items and
Register Sample Sort (Sec. 3) for segments of up to 256 items, behind the C
ABI of ``include/smallsort.h`` (``libsmallsort.so``).

This package is the thin Python binding of that library: argument marshalling
only, every sorting step runs in the CUDA kernels.  Functions take CUDA
tensors (or raw device addresses) and return the library's status code.
"""
from ._binding import (  # noqa: F401
    SN_EINVAL,
    SN_ENOMEM,
    SN_ERANGE,
    SN_ECUDA,
    SN_ETIMEOUT,
    SN_EUNSUPPORTED,
    SN_MAX_SEGMENT_LARGE,
    SN_NETWORK_BEST,
    SN_NETWORK_BOSE_NELSON,
    SN_OK,
    SmallSortError,
    SnTuning,
    check,
    library,
    library_path,
    rss_sort_segments,
    rss_sort_segments_u64,
    sn_check,
    sn_get_last_cuda_error,
    sn_sort_fixed,
    sn_sort_fixed_f32,
    sn_sort_fixed_f64,
    sn_sort_fixed_family,
    sn_sort_fixed_items,
    sn_sort_fixed_u64,
    sn_sort_large,
    sn_sort_segments,
    sn_sort_segments_f32,
    sn_sort_segments_f64,
    sn_sort_segments_large,
    sn_sort_segments_large_u64,
    sn_sort_segments_u64,
    sn_status_string,
    sn_tune,
    sn_tune_segments,
    sn_tuning_get,
    sn_tuning_load,
    sn_tuning_save,
    sn_tuning_set,
)
