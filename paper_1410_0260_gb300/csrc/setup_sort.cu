// Segmented and global sorts used by the setup stages (tree splits, node
// neighbor lists, work-list grouping).  Thin wrappers over CUB so the rest of
// the library compiles without its headers.  With tmp == nullptr each call
// only reports the scratch size it needs in *tmp_bytes.
#include <cub/cub.cuh>

#include "askit_impl.cuh"

#define CUB_CALL(expr)                                                               \
    do {                                                                             \
        cudaError_t e_ = (expr);                                                     \
        if (e_ != cudaSuccess) {                                                     \
            askit_set_error("%s:%d CUB: %s", __FILE__, __LINE__, cudaGetErrorString(e_)); \
            return ASKIT_ERR_CUDA;                                                   \
        }                                                                            \
    } while (0)

askit_status seg_sort_f64_i32(const double *kin, double *kout, const int32_t *vin, int32_t *vout,
                              int64_t n, int nseg, const int32_t *beg, const int32_t *end,
                              void *tmp, size_t *tmp_bytes, cudaStream_t s) {
    CUB_CALL(cub::DeviceSegmentedSort::StableSortPairs(tmp, *tmp_bytes, kin, kout, vin, vout,
                                                       (int)n, nseg, beg, end, s));
    return ASKIT_OK;
}

askit_status seg_sort_i32_f64(const int32_t *kin, int32_t *kout, const double *vin, double *vout,
                              int64_t n, int nseg, const int32_t *beg, const int32_t *end,
                              void *tmp, size_t *tmp_bytes, cudaStream_t s) {
    CUB_CALL(cub::DeviceSegmentedSort::StableSortPairs(tmp, *tmp_bytes, kin, kout, vin, vout,
                                                       (int)n, nseg, beg, end, s));
    return ASKIT_OK;
}

askit_status seg_sort_i32(const int32_t *kin, int32_t *kout, int64_t n, int nseg,
                          const int32_t *beg, const int32_t *end, void *tmp, size_t *tmp_bytes,
                          cudaStream_t s) {
    CUB_CALL(cub::DeviceSegmentedSort::StableSortKeys(tmp, *tmp_bytes, kin, kout, (int)n, nseg,
                                                      beg, end, s));
    return ASKIT_OK;
}

askit_status sort_u64_i32(const uint64_t *kin, uint64_t *kout, const int32_t *vin, int32_t *vout,
                          int64_t n, void *tmp, size_t *tmp_bytes, cudaStream_t s) {
    CUB_CALL(cub::DeviceRadixSort::SortPairs(tmp, *tmp_bytes, kin, kout, vin, vout, (int64_t)n, 0, 64, s));
    return ASKIT_OK;
}

askit_status sort_u64_i64(const uint64_t *kin, uint64_t *kout, const int64_t *vin, int64_t *vout,
                          int64_t n, void *tmp, size_t *tmp_bytes, cudaStream_t s) {
    CUB_CALL(cub::DeviceRadixSort::SortPairs(tmp, *tmp_bytes, kin, kout, vin, vout, (int64_t)n, 0, 64, s));
    return ASKIT_OK;
}

askit_status scan_i64(const int64_t *in, int64_t *out, int64_t n, void *tmp, size_t *tmp_bytes,
                      cudaStream_t s) {
    CUB_CALL(cub::DeviceScan::ExclusiveSum(tmp, *tmp_bytes, in, out, (int64_t)n, s));
    return ASKIT_OK;
}
