// ICON's nproma blocking of the state (Sec. 4.3: the model passes its own
// arrays): a Fortran array X(nproma, nlev_x, nblks) holds point h = jb nproma
// + jc (0-based jc, jb) at level k at offset jc + nproma (k + nlev_x jb),
// horizontal index fastest.  The library's layout is level-contiguous,
// X[h nlev_x + k].  These kernels convert between the two on the device with a
// shared-memory tiled transpose (coalesced on both sides); pad points of the
// last block (h >= n) are not read on import and not written on export.
#include <cuda_runtime.h>

#include "kernels.h"

namespace icon {
namespace {

constexpr int kTB = 32;  // tile edge (points x levels)

// to_blocked = false: blocked -> level-contiguous; true: the reverse
template <bool kToBlocked>
__global__ void blocked_transpose(int n, int nlev_x, int nproma, const double* __restrict__ src,
                                  double* __restrict__ dst) {
  __shared__ double tile[kTB][kTB + 1];
  const int jb = blockIdx.z;
  const int jc0 = blockIdx.x * kTB, k0 = blockIdx.y * kTB;
  const size_t bbase = (size_t)jb * nproma * nlev_x;  // start of block jb in the blocked array
  // load: threads x along the contiguous index of the source
  for (int r = threadIdx.y; r < kTB; r += blockDim.y) {
    if (!kToBlocked) {  // source blocked: contiguous in jc; r runs over levels
      const int jc = jc0 + threadIdx.x, k = k0 + r;
      const int h = jb * nproma + jc;
      if (jc < nproma && k < nlev_x && h < n) tile[r][threadIdx.x] = src[bbase + (size_t)k * nproma + jc];
    } else {  // source level-contiguous: contiguous in k; r runs over points
      const int jc = jc0 + r, k = k0 + threadIdx.x;
      const int h = jb * nproma + jc;
      if (jc < nproma && k < nlev_x && h < n) tile[threadIdx.x][r] = src[(size_t)h * nlev_x + k];
    }
  }
  __syncthreads();
  for (int r = threadIdx.y; r < kTB; r += blockDim.y) {
    if (!kToBlocked) {  // destination level-contiguous: contiguous in k; r runs over points
      const int jc = jc0 + r, k = k0 + threadIdx.x;
      const int h = jb * nproma + jc;
      if (jc < nproma && k < nlev_x && h < n) dst[(size_t)h * nlev_x + k] = tile[threadIdx.x][r];
    } else {  // destination blocked: contiguous in jc; r runs over levels
      const int jc = jc0 + threadIdx.x, k = k0 + r;
      const int h = jb * nproma + jc;
      if (jc < nproma && k < nlev_x && h < n) dst[bbase + (size_t)k * nproma + jc] = tile[r][threadIdx.x];
    }
  }
}

}  // namespace

void launch_blocked(bool to_blocked, int n, int nlev_x, int nproma, const double* src, double* dst, cudaStream_t s) {
  const int nblks = (n + nproma - 1) / nproma;
  dim3 grid((unsigned)((nproma + kTB - 1) / kTB), (unsigned)((nlev_x + kTB - 1) / kTB), (unsigned)nblks);
  dim3 block(kTB, 8);
  if (to_blocked)
    ICON_LAUNCH("blocked_export", grid, block, s, blocked_transpose<true>, n, nlev_x, nproma, src, dst);
  else
    ICON_LAUNCH("blocked_import", grid, block, s, blocked_transpose<false>, n, nlev_x, nproma, src, dst);
}

}  // namespace icon
