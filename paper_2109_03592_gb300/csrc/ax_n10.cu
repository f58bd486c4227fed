// Local-operator kernels instantiated for polynomial orders 10.
// (One translation unit per order keeps the parallel build short.)
#include "ax_eo_impl.cuh"
#include "ax_impl.cuh"

namespace sem {

cudaError_t ax64_n10(int v, bool f, const AxParams<double>& p, cudaStream_t s, int* g) {
  return dispatch_ax_n<double, 10>(v, f, p, s, g);
}
cudaError_t ax32_n10(int v, bool f, const AxParams<float>& p, cudaStream_t s, int* g) {
  return dispatch_ax_n<float, 10>(v, f, p, s, g);
}
cudaError_t axdf_n10(int v, bool f, const AxDFParams& p, cudaStream_t s, int* g) {
  return dispatch_fp64df_n<10>(v, f, p, s, g);
}

}  // namespace sem
