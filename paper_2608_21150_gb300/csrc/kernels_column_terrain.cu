// Row A7 over terrain: launches of the terrain-following forms of the column
// solve (kernel template in column_kernel.cuh): per-column metrics and the
// solve in the contravariant velocity w - wcc.
#include <cuda_runtime.h>

#include <type_traits>

#include "column_kernel.cuh"

namespace icon {

cudaError_t init_column_terrain_kernels() {
  cudaError_t e = init_col_forms<double, double, true>();
  if (e == cudaSuccess) e = init_col_forms<float, dws, true>();
  if (e == cudaSuccess) e = init_col_forms<float, double, true>();
  return e;
}

template <class T>
void launch_column_terrain(const Engine& en, int corrector, const StateView& st, const T* ddt_w0, const T* ddt_w1,
                           const T* wcc, cudaStream_t s) {
  ColArgs<T> a = col_args<T>(en, corrector, st, ddt_w0, ddt_w1);
  a.wcc = wcc;
  constexpr bool mixed = std::is_same<T, float>::value;
  const bool f64col = mixed && en.precision == ICON_PREC_MIXED_F64COL;
  const char* name = column_name(mixed, f64col, true, corrector);
  if (f64col)
    launch_col_form<T, double, true>(en, corrector, a, name, s);
  else
    launch_col_form<T, ColArith<T>, true>(en, corrector, a, name, s);
}

template void launch_column_terrain<double>(const Engine&, int, const StateView&, const double*, const double*,
                                            const double*, cudaStream_t);
template void launch_column_terrain<float>(const Engine&, int, const StateView&, const float*, const float*,
                                           const float*, cudaStream_t);

}  // namespace icon
