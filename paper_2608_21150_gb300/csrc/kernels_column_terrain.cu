// Row A7 over terrain: launches of the terrain-following forms of the column
// solve (kernel template in column_kernel.cuh): per-column metrics and the
// solve in the contravariant velocity w - wcc.
#include <cuda_runtime.h>

#include <type_traits>

#include "column_kernel.cuh"

namespace icon {

cudaError_t init_column_terrain_kernels() {
  cudaError_t e = cudaSuccess;
  auto set = [&](auto kernel, size_t bytes) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  };
  set(sn_column_tiled<double, false, 8, double, 0, true>, smem_bytes<double, 8, false, true>());
  set(sn_column_tiled<double, false, 8, double, 1, true>, smem_bytes<double, 8, true, true>());
  set(sn_column_tiled<float, false, 8, dws, 0, true>, smem_bytes<float, 8, false, true>());
  set(sn_column_tiled<float, false, 8, dws, 1, true>, smem_bytes<float, 8, true, true>());
  set(sn_column_tiled<double, false, 6, double, 0, true>, smem_bytes<double, 6, false, true>());
  set(sn_column_tiled<double, false, 6, double, 1, true>, smem_bytes<double, 6, true, true>());
  set(sn_column_tiled<float, false, 6, dws, 0, true>, smem_bytes<float, 6, false, true>());
  set(sn_column_tiled<float, false, 6, dws, 1, true>, smem_bytes<float, 6, true, true>());
  set(sn_column_tiled<double, false, 4, double, 0, true>, smem_bytes<double, 4, false, true>());
  set(sn_column_tiled<double, false, 4, double, 1, true>, smem_bytes<double, 4, true, true>());
  set(sn_column_tiled<float, false, 4, dws, 0, true>, smem_bytes<float, 4, false, true>());
  set(sn_column_tiled<float, false, 4, dws, 1, true>, smem_bytes<float, 4, true, true>());
  return e;
}

template <class T>
void launch_column_terrain(const Engine& en, int corrector, const StateView& st, const T* ddt_w0, const T* ddt_w1,
                           const T* wcc, cudaStream_t s) {
  ColArgs<T> a = col_args<T>(en, corrector, st, ddt_w0, ddt_w1);
  a.wcc = wcc;
  constexpr bool mixed = std::is_same<T, float>::value;
  const unsigned blocks = (unsigned)((en.g64.nc + kCW - 1) / kCW);
  const char* name = mixed ? (corrector ? "sn_column_corr_terrain_mx" : "sn_column_pred_terrain_mx")
                           : (corrector ? "sn_column_corr_terrain" : "sn_column_pred_terrain");
  using RA = ColArith<T>;
  const int nc = en.g64.nc;
  switch (en.col_kc * 2 + (corrector ? 1 : 0)) {
    case 6 * 2 + 1:
      ICON_LAUNCH_SMEM(name, blocks, kCW, (smem_bytes<T, 6, true, true>()), s, (sn_column_tiled<T, false, 6, RA, 1, true>),
                       nc, en.v, en.sc, 1, a);
      break;
    case 6 * 2:
      ICON_LAUNCH_SMEM(name, blocks, kCW, (smem_bytes<T, 6, false, true>()), s, (sn_column_tiled<T, false, 6, RA, 0, true>),
                       nc, en.v, en.sc, 0, a);
      break;
    case 4 * 2 + 1:
      ICON_LAUNCH_SMEM(name, blocks, kCW, (smem_bytes<T, 4, true, true>()), s, (sn_column_tiled<T, false, 4, RA, 1, true>),
                       nc, en.v, en.sc, 1, a);
      break;
    case 4 * 2:
      ICON_LAUNCH_SMEM(name, blocks, kCW, (smem_bytes<T, 4, false, true>()), s, (sn_column_tiled<T, false, 4, RA, 0, true>),
                       nc, en.v, en.sc, 0, a);
      break;
    case 8 * 2 + 1:
      ICON_LAUNCH_SMEM(name, blocks, kCW, (smem_bytes<T, 8, true, true>()), s, (sn_column_tiled<T, false, 8, RA, 1, true>),
                       nc, en.v, en.sc, 1, a);
      break;
    default:
      ICON_LAUNCH_SMEM(name, blocks, kCW, (smem_bytes<T, 8, false, true>()), s, (sn_column_tiled<T, false, 8, RA, 0, true>),
                       nc, en.v, en.sc, 0, a);
      break;
  }
}

template void launch_column_terrain<double>(const Engine&, int, const StateView&, const double*, const double*,
                                            const double*, cudaStream_t);
template void launch_column_terrain<float>(const Engine&, int, const StateView&, const float*, const float*,
                                           const float*, cudaStream_t);

}  // namespace icon
