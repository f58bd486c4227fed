// Local-operator kernels instantiated for polynomial orders 8.
// (One translation unit per order keeps the parallel build short.)
#include "ax_eo_impl.cuh"
#include "ax_impl.cuh"

namespace sem {

cudaError_t ax64_n8(int v, bool f, const AxParams<double>& p, cudaStream_t s, int* g) {
  return dispatch_ax_n<double, 8>(v, f, p, s, g);
}
cudaError_t ax32_n8(int v, bool f, const AxParams<float>& p, cudaStream_t s, int* g) {
  return dispatch_ax_n<float, 8>(v, f, p, s, g);
}
cudaError_t axdf_n8(int v, bool f, const AxDFParams& p, cudaStream_t s, int* g) {
  return dispatch_fp64df_n<8>(v, f, p, s, g);
}

}  // namespace sem
