// Dispatch of the local-operator kernels by polynomial order.
#include "kernels.h"

namespace sem {

cudaError_t ax64_n1(int, bool, const AxParams<double>&, cudaStream_t, int*);
cudaError_t ax32_n1(int, bool, const AxParams<float>&, cudaStream_t, int*);
cudaError_t axdf_n1(int, bool, const AxDFParams&, cudaStream_t, int*);
cudaError_t ax64_n2(int, bool, const AxParams<double>&, cudaStream_t, int*);
cudaError_t ax32_n2(int, bool, const AxParams<float>&, cudaStream_t, int*);
cudaError_t axdf_n2(int, bool, const AxDFParams&, cudaStream_t, int*);
cudaError_t ax64_n3(int, bool, const AxParams<double>&, cudaStream_t, int*);
cudaError_t ax32_n3(int, bool, const AxParams<float>&, cudaStream_t, int*);
cudaError_t axdf_n3(int, bool, const AxDFParams&, cudaStream_t, int*);
cudaError_t ax64_n4(int, bool, const AxParams<double>&, cudaStream_t, int*);
cudaError_t ax32_n4(int, bool, const AxParams<float>&, cudaStream_t, int*);
cudaError_t axdf_n4(int, bool, const AxDFParams&, cudaStream_t, int*);
cudaError_t ax64_n5(int, bool, const AxParams<double>&, cudaStream_t, int*);
cudaError_t ax32_n5(int, bool, const AxParams<float>&, cudaStream_t, int*);
cudaError_t axdf_n5(int, bool, const AxDFParams&, cudaStream_t, int*);
cudaError_t ax64_n6(int, bool, const AxParams<double>&, cudaStream_t, int*);
cudaError_t ax32_n6(int, bool, const AxParams<float>&, cudaStream_t, int*);
cudaError_t axdf_n6(int, bool, const AxDFParams&, cudaStream_t, int*);
cudaError_t ax64_n7(int, bool, const AxParams<double>&, cudaStream_t, int*);
cudaError_t ax32_n7(int, bool, const AxParams<float>&, cudaStream_t, int*);
cudaError_t axdf_n7(int, bool, const AxDFParams&, cudaStream_t, int*);
cudaError_t ax64_n8(int, bool, const AxParams<double>&, cudaStream_t, int*);
cudaError_t ax32_n8(int, bool, const AxParams<float>&, cudaStream_t, int*);
cudaError_t axdf_n8(int, bool, const AxDFParams&, cudaStream_t, int*);
cudaError_t ax64_n9(int, bool, const AxParams<double>&, cudaStream_t, int*);
cudaError_t ax32_n9(int, bool, const AxParams<float>&, cudaStream_t, int*);
cudaError_t axdf_n9(int, bool, const AxDFParams&, cudaStream_t, int*);
cudaError_t ax64_n10(int, bool, const AxParams<double>&, cudaStream_t, int*);
cudaError_t ax32_n10(int, bool, const AxParams<float>&, cudaStream_t, int*);
cudaError_t axdf_n10(int, bool, const AxDFParams&, cudaStream_t, int*);
cudaError_t ax64_n11(int, bool, const AxParams<double>&, cudaStream_t, int*);
cudaError_t ax32_n11(int, bool, const AxParams<float>&, cudaStream_t, int*);
cudaError_t axdf_n11(int, bool, const AxDFParams&, cudaStream_t, int*);

int ax_num_variants() { return 4; }

int ax_elems_per_block(int N, int variant) {
  const int t = (variant == 0 || variant == 3) ? 256 : 128, per = (N + 1) * (N + 1);
  return t / per < 1 ? 1 : t / per;
}

int ax_df_available(int N) { return N >= 1 && N <= 11; }

cudaError_t launch_ax_f64(int N, int variant, bool fused, const AxParams<double>& p, cudaStream_t s, int* grid_out) {
  switch (N) {
    case 1: return ax64_n1(variant, fused, p, s, grid_out);
    case 2: return ax64_n2(variant, fused, p, s, grid_out);
    case 3: return ax64_n3(variant, fused, p, s, grid_out);
    case 4: return ax64_n4(variant, fused, p, s, grid_out);
    case 5: return ax64_n5(variant, fused, p, s, grid_out);
    case 6: return ax64_n6(variant, fused, p, s, grid_out);
    case 7: return ax64_n7(variant, fused, p, s, grid_out);
    case 8: return ax64_n8(variant, fused, p, s, grid_out);
    case 9: return ax64_n9(variant, fused, p, s, grid_out);
    case 10: return ax64_n10(variant, fused, p, s, grid_out);
    case 11: return ax64_n11(variant, fused, p, s, grid_out);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_ax_f32(int N, int variant, bool fused, const AxParams<float>& p, cudaStream_t s, int* grid_out) {
  switch (N) {
    case 1: return ax32_n1(variant, fused, p, s, grid_out);
    case 2: return ax32_n2(variant, fused, p, s, grid_out);
    case 3: return ax32_n3(variant, fused, p, s, grid_out);
    case 4: return ax32_n4(variant, fused, p, s, grid_out);
    case 5: return ax32_n5(variant, fused, p, s, grid_out);
    case 6: return ax32_n6(variant, fused, p, s, grid_out);
    case 7: return ax32_n7(variant, fused, p, s, grid_out);
    case 8: return ax32_n8(variant, fused, p, s, grid_out);
    case 9: return ax32_n9(variant, fused, p, s, grid_out);
    case 10: return ax32_n10(variant, fused, p, s, grid_out);
    case 11: return ax32_n11(variant, fused, p, s, grid_out);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_ax_df(int N, int variant, bool fused, const AxDFParams& p, cudaStream_t s, int* grid_out) {
  switch (N) {
    case 1: return axdf_n1(variant, fused, p, s, grid_out);
    case 2: return axdf_n2(variant, fused, p, s, grid_out);
    case 3: return axdf_n3(variant, fused, p, s, grid_out);
    case 4: return axdf_n4(variant, fused, p, s, grid_out);
    case 5: return axdf_n5(variant, fused, p, s, grid_out);
    case 6: return axdf_n6(variant, fused, p, s, grid_out);
    case 7: return axdf_n7(variant, fused, p, s, grid_out);
    case 8: return axdf_n8(variant, fused, p, s, grid_out);
    case 9: return axdf_n9(variant, fused, p, s, grid_out);
    case 10: return axdf_n10(variant, fused, p, s, grid_out);
    case 11: return axdf_n11(variant, fused, p, s, grid_out);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace sem
