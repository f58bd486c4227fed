// Local-operator kernels instantiated for polynomial orders 1, 2, 3, 4.
// (One translation unit per order keeps the parallel build short.)
#include "ax_eo_impl.cuh"
#include "ax_impl.cuh"

namespace sem {

cudaError_t ax64_n1(int v, bool f, const AxParams<double>& p, cudaStream_t s, int* g) {
  return dispatch_ax_n<double, 1>(v, f, p, s, g);
}
cudaError_t ax32_n1(int v, bool f, const AxParams<float>& p, cudaStream_t s, int* g) {
  return dispatch_ax_n<float, 1>(v, f, p, s, g);
}
cudaError_t axdf_n1(int v, bool f, const AxDFParams& p, cudaStream_t s, int* g) {
  return dispatch_fp64df_n<1>(v, f, p, s, g);
}

cudaError_t ax64_n2(int v, bool f, const AxParams<double>& p, cudaStream_t s, int* g) {
  return dispatch_ax_n<double, 2>(v, f, p, s, g);
}
cudaError_t ax32_n2(int v, bool f, const AxParams<float>& p, cudaStream_t s, int* g) {
  return dispatch_ax_n<float, 2>(v, f, p, s, g);
}
cudaError_t axdf_n2(int v, bool f, const AxDFParams& p, cudaStream_t s, int* g) {
  return dispatch_fp64df_n<2>(v, f, p, s, g);
}

cudaError_t ax64_n3(int v, bool f, const AxParams<double>& p, cudaStream_t s, int* g) {
  return dispatch_ax_n<double, 3>(v, f, p, s, g);
}
cudaError_t ax32_n3(int v, bool f, const AxParams<float>& p, cudaStream_t s, int* g) {
  return dispatch_ax_n<float, 3>(v, f, p, s, g);
}
cudaError_t axdf_n3(int v, bool f, const AxDFParams& p, cudaStream_t s, int* g) {
  return dispatch_fp64df_n<3>(v, f, p, s, g);
}

cudaError_t ax64_n4(int v, bool f, const AxParams<double>& p, cudaStream_t s, int* g) {
  return dispatch_ax_n<double, 4>(v, f, p, s, g);
}
cudaError_t ax32_n4(int v, bool f, const AxParams<float>& p, cudaStream_t s, int* g) {
  return dispatch_ax_n<float, 4>(v, f, p, s, g);
}
cudaError_t axdf_n4(int v, bool f, const AxDFParams& p, cudaStream_t s, int* g) {
  return dispatch_fp64df_n<4>(v, f, p, s, g);
}

}  // namespace sem
