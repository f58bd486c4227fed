// Local-operator kernels instantiated for polynomial orders 11.
// (One translation unit per order keeps the parallel build short.)
#include "ax_eo_impl.cuh"
#include "ax_impl.cuh"

namespace sem {

cudaError_t ax64_n11(int v, bool f, const AxParams<double>& p, cudaStream_t s, int* g) {
  return dispatch_ax_n<double, 11>(v, f, p, s, g);
}
cudaError_t ax32_n11(int v, bool f, const AxParams<float>& p, cudaStream_t s, int* g) {
  return dispatch_ax_n<float, 11>(v, f, p, s, g);
}
cudaError_t axdf_n11(int v, bool f, const AxDFParams& p, cudaStream_t s, int* g) {
  return dispatch_fp64df_n<11>(v, f, p, s, g);
}

}  // namespace sem
