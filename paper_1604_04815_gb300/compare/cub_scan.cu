// cub_scan.cu -- a comparator for the benchmark, not part of the scan
// library: CUB's single-pass device scan (cub::DeviceScan, compiled from the
// CUDA toolkit's CUB headers) on the same buffers bench.py times this
// library's kernels on.  CUB's scan is a decoupled look-back scan (the same
// family as Section 4.3's inter-block carry), so it is the natural external
// reference point for a single-pass scan on one GPU.  Built into its own
// shared library (libcubcmp.so); liblscan.so does not link or call it.
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <cub/device/device_scan.cuh>
#include <cuda/functional>

namespace {

// op: 0 add, 1 max; dtype: 0 int32, 1 fp32 (the benchmark's types)
template <class T>
cudaError_t scan_t(int op, const void *x, void *y, int n, void *tmp, size_t *bytes,
                   cudaStream_t s) {
    const T *in = static_cast<const T *>(x);
    T *out = static_cast<T *>(y);
    if (op == 0) return cub::DeviceScan::InclusiveSum(tmp, *bytes, in, out, n, s);
    return cub::DeviceScan::InclusiveScan(tmp, *bytes, in, out, cuda::maximum<>{}, n, s);
}

cudaError_t dispatch(int op, int dtype, const void *x, void *y, long long n, void *tmp,
                     size_t *bytes, cudaStream_t s) {
    if (n < 0 || n > 0x7fffffffLL || (op != 0 && op != 1)) return cudaErrorInvalidValue;
    const int ni = static_cast<int>(n);
    if (dtype == 0) return scan_t<int32_t>(op, x, y, ni, tmp, bytes, s);
    if (dtype == 1) return scan_t<float>(op, x, y, ni, tmp, bytes, s);
    return cudaErrorInvalidValue;
}

}  // namespace

extern "C" {

// Bytes of temporary device storage an inclusive scan of n elements needs
// (written to *bytes); returns a cudaError_t value (0 on success).
int cubcmp_temp_bytes(int op, int dtype, long long n, size_t *bytes) {
    if (bytes == nullptr) return static_cast<int>(cudaErrorInvalidValue);
    *bytes = 0;
    return static_cast<int>(dispatch(op, dtype, nullptr, nullptr, n, nullptr, bytes, nullptr));
}

// Inclusive scan of n elements of x into y on `stream` with caller-owned
// temporary storage of temp_bytes (at least cubcmp_temp_bytes); returns a
// cudaError_t value.  x, y, temp: device pointers.
int cubcmp_inclusive(int op, int dtype, const void *x, void *y, long long n, void *temp,
                     size_t temp_bytes, void *stream) {
    if (temp == nullptr) return static_cast<int>(cudaErrorInvalidValue);
    size_t b = temp_bytes;
    return static_cast<int>(
        dispatch(op, dtype, x, y, n, temp, &b, static_cast<cudaStream_t>(stream)));
}

}  // extern "C"
