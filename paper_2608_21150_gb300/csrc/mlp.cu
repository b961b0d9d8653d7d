// Learned corrector (row A13): a 3-layer MLP, x -> GELU(x W1 + b1) -> GELU(. W2 + b2)
// -> . W3 + b3, with BF16 weights and activations and FP32 accumulation on the
// tensor cores, plus its backward pass and an Adam update for training on the
// GPU.  GELU is the erf form, 0.5 x (1 + erf(x / sqrt(2))).
//
// Every GEMM is C[M x N] = A[M x K] * B[N x K]^T with both operands K-major
// ("NT"), the layout tcgen05.mma reads from 128-byte-swizzled shared memory
// without transposes.  Leading dimensions are padded to multiples of 64 and
// the pads hold zeros, so K needs no tail handling; rows of A and B past M and
// N read as zero through the TMA bounds and the epilogue stores guard them.
// The backward GEMMs reuse the same kernel on transposed copies (dW^T = dZ^T
// H over the batch, dH = dZ W).  The forward epilogue's GELU uses a 1.5e-7
// erf approximation (below); the backward pass differentiates the erf form.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "mlp.h"

namespace icon {
namespace {

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
  // d/dx [x Phi(x)] = Phi(x) + x phi(x)
  const float cdf = 0.5f * (1.0f + erff(x * 0.70710678118654752f));
  const float pdf = 0.3989422804014327f * expf(-0.5f * x * x);
  return cdf + x * pdf;
}

// GELU for the forward epilogue, with erf from Abramowitz & Stegun, Handbook of
// Mathematical Functions, formula 7.1.26 (|error| <= 1.5e-7, far below the
// BF16 rounding of the stored activation): erf(x) = 1 - (a1 t + ... + a5 t^5)
// exp(-x^2), t = 1/(1 + p x), x >= 0, odd extension.
__device__ __forceinline__ float gelu_fwd(float x) {
  const float z = fabsf(x) * 0.70710678118654752f;
  const float t = __fdividef(1.0f, fmaf(0.3275911f, z, 1.0f));
  const float poly =
      t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, 1.061405429f, -1.453152027f), 1.421413741f), -0.284496736f), 0.254829592f);
  const float e = 1.0f - poly * __expf(-z * z);
  return 0.5f * x * (1.0f + copysignf(e, x));
}

// ---------------------------------------------------------------------------
// Tensor-core GEMM (tcgen05), persistent and warp-specialised.  Each CTA (one
// per SM, 170 KB of shared memory) walks output tiles of 128 x 128 (N
// fastest, so the CTAs in flight share A rows in L2); K runs in blocks of 64
// BF16 (one 128-byte swizzle row) through a 5-stage TMA ring that continues
// across tiles.  Warp 0 (one lane) issues the TMA loads; warp 1 (one lane) the
// MMAs, into one of two 128-column FP32 accumulators in tensor memory; warps
// 2..9 drain the other accumulator meanwhile (TMEM -> registers -> bias, GELU,
// stores): warp w may access TMEM lanes 32 (w % 4) .. +31 (= tile rows), and
// the two warps of a lane quarter split the columns.
constexpr int TBM = 128, TBN = 128, TBK = 64, kStages = 5;
constexpr int kEpiWarps = 8;
constexpr int kTcThreads = 64 + 32 * kEpiWarps;
constexpr int kTileBytesA = TBM * TBK * 2, kTileBytesB = TBN * TBK * 2;
// per epilogue warp, a staging block of its 32 rows x 64 columns of BF16 output
constexpr int kStageBytes = 32 * 64 * 2;
constexpr int kTcSmem = kStages * (kTileBytesA + kTileBytesB) + kEpiWarps * kStageBytes +
                        1024 /* alignment slack */ + 256 /* barriers */;
constexpr uint32_t kTmemCols = 2 * TBN;
// every wait gives up after this long (ns) and flags an error instead of hanging
constexpr unsigned long long kWaitLimitNs = 1000000000ull;

__device__ int g_tc_error = 0;

// Epilogue modes: 0 = fp32 out (+bias if given); 1 = bias + GELU -> bf16 out,
// fp32 pre-activation stored if zpre != null.
struct Epi {
  int mode;
  const float* bias;  // [N] or null
  float* out_f32;     // mode 0
  __nv_bfloat16* out_bf16;  // mode 1
  float* zpre;        // mode 1, optional
  int ldc;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the completion of the phase with the given parity.  Gives up
// when another thread of the CTA has flagged an abort, or after kWaitLimitNs
// (then flags the abort and the device-wide error word itself).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  const unsigned long long t0 = now_ns();
  for (uint32_t i = 0;; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 255u) == 255u) {
      if (*abort_flag) return false;
      if (now_ns() - t0 > kWaitLimitNs) {
        *abort_flag = 1;
        atomicExch(&g_tc_error, 1);
        return false;
      }
    }
  }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major operand tile stored as rows of
// 128 bytes with the 128-byte swizzle (as TMA writes it): start address,
// stride between 8-row groups 1024 B, descriptor version 1, swizzle mode 2.
// The leading-byte offset is unused for this layout.
__device__ __forceinline__ uint64_t sdesc_sw128(const void* tile) {
  const uint32_t a = smem_u32(tile);
  return (uint64_t)((a & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16_tc(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// Epilogue of one 16-column run of a tile row (thread-private values v).
__device__ __forceinline__ void epilogue16(float (&v)[16], int row, int col0, int M, int N, const Epi& ep) {
  if (row >= M || col0 >= N) return;
  const bool whole = col0 + 16 <= N;
  const size_t o = (size_t)row * ep.ldc + col0;
  const bool vec32 = whole && (o & 3) == 0;  // 16-byte aligned fp32 run
  const bool vec16 = whole && (o & 7) == 0;  // 16-byte aligned bf16 run
  if (ep.bias) {
    if (whole) {
      const float4* b4 = reinterpret_cast<const float4*>(ep.bias + col0);  // col0 % 16 == 0, bias 16-byte aligned
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 bq = __ldg(b4 + q);
        v[4 * q] += bq.x;
        v[4 * q + 1] += bq.y;
        v[4 * q + 2] += bq.z;
        v[4 * q + 3] += bq.w;
      }
    } else {
      for (int j = 0; j < 16 && col0 + j < N; ++j) v[j] += ep.bias[col0 + j];
    }
  }
  if (ep.mode == 0) {
    if (vec32) {
      float4* dst = reinterpret_cast<float4*>(ep.out_f32 + o);
#pragma unroll
      for (int q = 0; q < 4; ++q) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    } else {
      for (int j = 0; j < 16 && col0 + j < N; ++j) ep.out_f32[o + j] = v[j];
    }
  } else {
    if (ep.zpre) {
      if (vec32) {
        float4* dst = reinterpret_cast<float4*>(ep.zpre + o);
#pragma unroll
        for (int q = 0; q < 4; ++q) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
      } else {
        for (int j = 0; j < 16 && col0 + j < N; ++j) ep.zpre[o + j] = v[j];
      }
    }
    if (vec16) {
      __align__(16) __nv_bfloat16 h[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) h[j] = __float2bfloat16(gelu_fwd(v[j]));
      uint4* dst = reinterpret_cast<uint4*>(ep.out_bf16 + o);
      dst[0] = reinterpret_cast<const uint4*>(h)[0];
      dst[1] = reinterpret_cast<const uint4*>(h)[1];
    } else {
      for (int j = 0; j < 16 && col0 + j < N; ++j) ep.out_bf16[o + j] = __float2bfloat16(gelu_fwd(v[j]));
    }
  }
}

__global__ void __launch_bounds__(kTcThreads, 1) gemm_tc(const __grid_constant__ CUtensorMap tma_a,
                                                         const __grid_constant__ CUtensorMap tma_b, int M, int N,
                                                         int K, Epi ep) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = base;
  uint8_t* sB = base + kStages * kTileBytesA;
  uint8_t* sOut = sB + kStages * kTileBytesB;  // the epilogue warps' staging blocks
  uint64_t* full = reinterpret_cast<uint64_t*>(sOut + kEpiWarps * kStageBytes);
  uint64_t* empty = full + kStages;
  uint64_t* acc_full = empty + kStages;   // [2] MMA -> epilogue
  uint64_t* acc_empty = acc_full + 2;     // [2] epilogue -> MMA
  uint64_t* drain = acc_empty + 2;        // MMA issuer's own completion wait
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tiles_n = (N + TBN - 1) / TBN;
  const int n_tiles = ((M + TBM - 1) / TBM) * tiles_n;
  const int nk = K / TBK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], kEpiWarps);
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  int issued = 0;  // k-blocks whose TMA loads the producer lane issued (all tiles)
  if (warp == 0 && lane == 0) {
    int g = 0;
    for (int tile = blockIdx.x; tile < n_tiles && !*abort_flag; tile += gridDim.x) {
      const int m0 = (tile / tiles_n) * TBM, n0 = (tile % tiles_n) * TBN;
      for (int kb = 0; kb < nk; ++kb, ++g) {
        const int s = g % kStages;
        if (g >= kStages && !mbar_wait(&empty[s], ((g / kStages) & 1) ^ 1, abort_flag)) break;
        mbar_expect_tx(&full[s], kTileBytesA + kTileBytesB);
        tma_load_2d(sA + s * kTileBytesA, &tma_a, kb * TBK, m0, &full[s]);
        tma_load_2d(sB + s * kTileBytesB, &tma_b, kb * TBK, n0, &full[s]);
        issued = g + 1;
      }
    }
  } else if (warp == 1 && lane == 0) {
    constexpr uint32_t idesc = idesc_bf16(TBM, TBN);
    int g = 0, t = 0;
    bool ok = true;
    for (int tile = blockIdx.x; ok && tile < n_tiles; tile += gridDim.x, ++t) {
      const int b = t & 1;
      const uint32_t d = tmem + (uint32_t)(b * TBN);
      if (t >= 2 && !mbar_wait(&acc_empty[b], ((t >> 1) & 1) ^ 1, abort_flag)) break;
      tc_fence_after();
      for (int kb = 0; kb < nk; ++kb, ++g) {
        const int s = g % kStages;
        if (!mbar_wait(&full[s], (g / kStages) & 1, abort_flag)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint64_t da = sdesc_sw128(sA + s * kTileBytesA), db = sdesc_sw128(sB + s * kTileBytesB);
#pragma unroll
        for (int k = 0; k < TBK / 16; ++k)  // 16 BF16 = 32 bytes further along K: +2 in the 16-byte address field
          mma_bf16_tc(d, da + 2 * k, db + 2 * k, idesc, (kb > 0 || k > 0) ? 1u : 0u);
        tc_commit(&empty[s]);
      }
      if (ok) tc_commit(&acc_full[b]);
    }
    // every MMA issued above has completed before the teardown frees TMEM
    tc_commit(drain);
    if (!mbar_wait(drain, 0, abort_flag)) {
      const unsigned long long t0 = now_ns();
      while (!mbar_try_wait(drain, 0) && now_ns() - t0 < kWaitLimitNs) {
      }
    }
  } else if (warp >= 2) {
    // epilogue: thread (warp, lane) owns tile row 32 (warp % 4) + lane and
    // half of the columns
    const int quarter = warp & 3, half = (warp - 2) >> 2;
    int t = 0;
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++t) {
      const int b = t & 1;
      // warp-uniform decision: the tcgen05.ld below is a warp-collective instruction
      if (!__all_sync(0xffffffffu, mbar_wait(&acc_full[b], (t >> 1) & 1, abort_flag))) break;
      tc_fence_after();
      const int m0 = (tile / tiles_n) * TBM, n0 = (tile % tiles_n) * TBN;
      const int row = m0 + 32 * quarter + lane;
      const uint32_t trow = tmem + (uint32_t)(b * TBN) + ((uint32_t)(32 * quarter) << 16);
      const int cw = n0 + half * (TBN / 2);  // first column of this warp's half
      if (ep.mode == 1 && !ep.zpre && cw + TBN / 2 <= N && (ep.ldc & 1) == 0 &&
          (reinterpret_cast<uintptr_t>(ep.out_bf16) & 3) == 0) {
        // GELU to BF16 staged in this warp's block (row = lane, 16-byte chunks
        // XOR-swizzled by the row so that 8 lanes writing one chunk hit all
        // banks), then stored row by row as 128-byte runs
        uint8_t* st = sOut + (warp - 2) * kStageBytes;
#pragma unroll 1
        for (int c = 0; c < TBN / 2; c += 16) {
          float v[16];
          tmem_ld16(trow + (uint32_t)(half * (TBN / 2) + c), v);
          if (ep.bias) {
            const float4* b4 = reinterpret_cast<const float4*>(ep.bias + cw + c);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const float4 bq = __ldg(b4 + q);
              v[4 * q] += bq.x;
              v[4 * q + 1] += bq.y;
              v[4 * q + 2] += bq.z;
              v[4 * q + 3] += bq.w;
            }
          }
          uint32_t h[8];  // BF16 pairs, the lower column in the low half
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const __nv_bfloat162 p2 = __floats2bfloat162_rn(gelu_fwd(v[2 * j]), gelu_fwd(v[2 * j + 1]));
            h[j] = *reinterpret_cast<const uint32_t*>(&p2);
          }
          const int ch = c / 8;  // logical 16-byte chunk of the row
          *reinterpret_cast<uint4*>(st + lane * 128 + ((ch ^ (lane & 7)) * 16)) = make_uint4(h[0], h[1], h[2], h[3]);
          *reinterpret_cast<uint4*>(st + lane * 128 + (((ch + 1) ^ (lane & 7)) * 16)) =
              make_uint4(h[4], h[5], h[6], h[7]);
        }
        __syncwarp();
#pragma unroll 4
        for (int r = 0; r < 32; ++r) {
          const int grow = m0 + 32 * quarter + r;
          const uint32_t val =
              *reinterpret_cast<const uint32_t*>(st + r * 128 + (((lane >> 2) ^ (r & 7)) * 16) + (lane & 3) * 4);
          if (grow < M) *reinterpret_cast<uint32_t*>(ep.out_bf16 + (size_t)grow * ep.ldc + cw + 2 * lane) = val;
        }
        __syncwarp();
      } else if (ep.mode == 0 && cw + TBN / 2 <= N) {
        // FP32 (+ bias) staged the same way, 32 columns (128 bytes a row) at a time
        uint8_t* st = sOut + (warp - 2) * kStageBytes;
#pragma unroll 1
        for (int c2 = 0; c2 < TBN / 2; c2 += 32) {
#pragma unroll
          for (int hh = 0; hh < 2; ++hh) {
            const int c = c2 + 16 * hh;
            float v[16];
            tmem_ld16(trow + (uint32_t)(half * (TBN / 2) + c), v);
            if (ep.bias) {
              const float4* b4 = reinterpret_cast<const float4*>(ep.bias + cw + c);
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                const float4 bq = __ldg(b4 + q);
                v[4 * q] += bq.x;
                v[4 * q + 1] += bq.y;
                v[4 * q + 2] += bq.z;
                v[4 * q + 3] += bq.w;
              }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int ch = 4 * hh + q;  // logical 16-byte chunk of the 128-byte row
              *reinterpret_cast<float4*>(st + lane * 128 + ((ch ^ (lane & 7)) * 16)) =
                  make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            }
          }
          __syncwarp();
#pragma unroll 4
          for (int r = 0; r < 32; ++r) {
            const int grow = m0 + 32 * quarter + r;
            const float val =
                *reinterpret_cast<const float*>(st + r * 128 + (((lane >> 2) ^ (r & 7)) * 16) + (lane & 3) * 4);
            if (grow < M) ep.out_f32[(size_t)grow * ep.ldc + cw + c2 + lane] = val;
          }
          __syncwarp();
        }
      } else {
#pragma unroll 1
        for (int c = half * (TBN / 2); c < (half + 1) * (TBN / 2); c += 16) {
          float v[16];
          tmem_ld16(trow + (uint32_t)c, v);
          epilogue16(v, row, n0 + c, M, N, ep);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[b]);
    }
  }

  // teardown: the TMA copies this CTA issued have landed (bounded), then TMEM is freed
  tc_fence_before();
  __syncthreads();
  if (warp == 0 && lane == 0 && *abort_flag) {
    const int first = issued > kStages ? issued - kStages : 0;
    for (int g = first; g < issued; ++g) {
      const unsigned long long t0 = now_ns();
      while (!mbar_try_wait(&full[g % kStages], (g / kStages) & 1) && now_ns() - t0 < kWaitLimitNs) {
      }
    }
  }
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

// out[c][r] = in[r][c] for r < rows, c < cols (bf16); pads of out left untouched
__global__ void transpose_bf16(int rows, int cols, const __nv_bfloat16* __restrict__ in, int ldi,
                               __nv_bfloat16* __restrict__ out, int ldo) {
  __shared__ __nv_bfloat16 tile[32][33];
  const int c = blockIdx.x * 32 + threadIdx.x, r0 = blockIdx.y * 32;
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int r = r0 + j;
    if (r < rows && c < cols) tile[j][threadIdx.x] = in[(size_t)r * ldi + c];
  }
  __syncthreads();
  const int rr = r0 + threadIdx.x;
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int cc = blockIdx.x * 32 + j;
    if (rr < rows && cc < cols) out[(size_t)cc * ldo + rr] = tile[threadIdx.x][j];
  }
}

// dZ = dH * gelu'(Z) (bf16 out for the next GEMMs, fp32 kept for the bias gradient)
__global__ void gelu_backward(int rows, int cols, const float* __restrict__ dh, int ldd,
                              const float* __restrict__ z, int ldz, float* __restrict__ dz32,
                              __nv_bfloat16* __restrict__ dz16, int ldo) {
  const size_t n = (size_t)rows * cols;
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int r = (int)(i / cols), c = (int)(i - (size_t)r * cols);
  const float v = dh[(size_t)r * ldd + c] * gelu_grad(z[(size_t)r * ldz + c]);
  dz32[(size_t)r * ldo + c] = v;
  dz16[(size_t)r * ldo + c] = __float2bfloat16(v);
}

// fp32 -> bf16 copy with padding (pads written as zero)
__global__ void to_bf16(int rows, int cols, const float* __restrict__ in, int ldi, __nv_bfloat16* __restrict__ out,
                        int ldo) {
  const size_t n = (size_t)rows * ldo;
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int r = (int)(i / ldo), c = (int)(i - (size_t)r * ldo);
  out[i] = __float2bfloat16(c < cols ? in[(size_t)r * ldi + c] : 0.f);
}

// db[c] = sum_r dz[r][c], fixed order per column (one thread per column)
__global__ void bias_grad(int rows, int cols, const float* __restrict__ dz, int ldd, float* __restrict__ db) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float s = 0.f;
  for (int r = 0; r < rows; ++r) s += dz[(size_t)r * ldd + c];
  db[c] = s;
}

// Adam on fp32 master weights; refreshes the bf16 copy W^T [n][k] and W [k][n]
__global__ void adam_update(int n_out, int n_in, float* __restrict__ w, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, float lr, float b1, float b2, float eps,
                            float c1, float c2, __nv_bfloat16* __restrict__ wt16, int ldt,
                            __nv_bfloat16* __restrict__ w16, int ldw) {
  const size_t n = (size_t)n_out * n_in;
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  w[i] = wi;
  if (wt16) {
    const int o = (int)(i / n_in), k = (int)(i - (size_t)o * n_in);
    wt16[(size_t)o * ldt + k] = __float2bfloat16(wi);
    w16[(size_t)k * ldw + o] = __float2bfloat16(wi);
  }
}

__global__ void adam_update_bias(int n, float* __restrict__ b, const float* __restrict__ g, float* __restrict__ m,
                                 float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  b[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

inline unsigned cdiv(size_t a, size_t b) { return (unsigned)((a + b - 1) / b); }

using EncodeTiled = PFN_cuTensorMapEncodeTiled_v12000;

EncodeTiled encode_tiled() {
  static EncodeTiled fn = []() -> EncodeTiled {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return reinterpret_cast<EncodeTiled>(p);
  }();
  return fn;
}

// 2-D tensor map of a K-major BF16 operand [rows][ld] (K of it used): boxes of
// 64 (K) x box_rows, 128-byte swizzle; rows past `rows` read as zero.
bool operand_map(CUtensorMap* map, const __nv_bfloat16* ptr, int rows, int K, int ld, int box_rows) {
  EncodeTiled enc = encode_tiled();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(__nv_bfloat16)};
  const cuuint32_t box[2] = {(cuuint32_t)TBK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(ptr), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

std::mutex g_attr_mutex;
bool g_attr_set[64] = {};
int g_sm_count[64] = {};

}  // namespace

int mlp_gemm(int M, int N, int K, const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb,
             const float* bias, bool gelu_act, float* out_f32, __nv_bfloat16* out_bf16, float* zpre, int ldc,
             cudaStream_t s) {
  if (M < 1 || N < 1 || K < TBK || K % TBK || lda % 8 || ldb % 8 || ldc < N || lda < K || ldb < K ||
      (reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B) | reinterpret_cast<uintptr_t>(bias)) % 16)
    return report_error(ICON_ERR_ARG, "mlp_gemm: unsupported shape or alignment");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return report_error(ICON_ERR_CUDA, "mlp_gemm: device");
  {
    std::lock_guard<std::mutex> lk(g_attr_mutex);
    if (!g_attr_set[dev]) {
      if (cudaFuncSetAttribute(gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem) != cudaSuccess)
        return report_error(ICON_ERR_CUDA, "mlp_gemm: shared memory attribute");
      if (cudaDeviceGetAttribute(&g_sm_count[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
          g_sm_count[dev] < 1)
        return report_error(ICON_ERR_CUDA, "mlp_gemm: SM count");
      g_attr_set[dev] = true;
    }
  }
  CUtensorMap ta, tb;
  if (!operand_map(&ta, A, M, K, lda, TBM) || !operand_map(&tb, B, N, K, ldb, TBN))
    return report_error(ICON_ERR_CUDA, "mlp_gemm: tensor map encoding failed");
  Epi ep{gelu_act ? 1 : 0, bias, out_f32, out_bf16, zpre, ldc};
  const long long tiles = (long long)cdiv(N, TBN) * cdiv(M, TBM);
  const unsigned grid = (unsigned)std::min<long long>(tiles, g_sm_count[dev]);  // one persistent CTA per SM
  ICON_LAUNCH_SMEM("mlp_gemm_tc", grid, kTcThreads, kTcSmem, s, gemm_tc, ta, tb, M, N, K, ep);
  return ICON_OK;
}

const int* mlp_tc_error_flag() {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_tc_error) != cudaSuccess) return nullptr;
  return static_cast<const int*>(p);
}

void mlp_transpose(int rows, int cols, const __nv_bfloat16* in, int ldi, __nv_bfloat16* out, int ldo,
                   cudaStream_t s) {
  dim3 grid(cdiv(cols, 32), cdiv(rows, 32));
  ICON_LAUNCH("mlp_transpose", grid, dim3(32, 8), s, transpose_bf16, rows, cols, in, ldi, out, ldo);
}

void mlp_gelu_backward(int rows, int cols, const float* dh, int ldd, const float* z, int ldz, float* dz32,
                       __nv_bfloat16* dz16, int ldo, cudaStream_t s) {
  ICON_LAUNCH("mlp_gelu_backward", cdiv((size_t)rows * cols, 256), 256, s, gelu_backward, rows, cols, dh, ldd, z,
              ldz, dz32, dz16, ldo);
}

void mlp_to_bf16(int rows, int cols, const float* in, int ldi, __nv_bfloat16* out, int ldo, cudaStream_t s) {
  ICON_LAUNCH("mlp_to_bf16", cdiv((size_t)rows * ldo, 256), 256, s, to_bf16, rows, cols, in, ldi, out, ldo);
}

void mlp_bias_grad(int rows, int cols, const float* dz, int ldd, float* db, cudaStream_t s) {
  ICON_LAUNCH("mlp_bias_grad", cdiv(cols, 128), 128, s, bias_grad, rows, cols, dz, ldd, db);
}

void mlp_adam(int n_out, int n_in, float* w, const float* g, float* m, float* v, float lr, float b1, float b2,
              float eps, float c1, float c2, __nv_bfloat16* wt16, int ldt, __nv_bfloat16* w16, int ldw,
              cudaStream_t s) {
  ICON_LAUNCH("mlp_adam", cdiv((size_t)n_out * n_in, 256), 256, s, adam_update, n_out, n_in, w, g, m, v, lr, b1, b2,
              eps, c1, c2, wt16, ldt, w16, ldw);
}

void mlp_adam_bias(int n, float* b, const float* g, float* m, float* v, float lr, float b1, float b2, float eps,
                   float c1, float c2, cudaStream_t s) {
  ICON_LAUNCH("mlp_adam_bias", cdiv(n, 256), 256, s, adam_update_bias, n, b, g, m, v, lr, b1, b2, eps, c1, c2);
}

}  // namespace icon

namespace icon {
namespace {
__global__ void mse_kernel(int B, int n_out, const float* __restrict__ y, int ldy, const float* __restrict__ t,
                           int ldt, float* __restrict__ dy, int lddy, double* __restrict__ rowloss) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= B) return;
  const float scale = 2.0f / ((float)B * (float)n_out);
  double s = 0.0;
  for (int c = 0; c < n_out; ++c) {
    const float d = y[(size_t)r * ldy + c] - t[(size_t)r * ldt + c];
    s += (double)d * d;
    dy[(size_t)r * lddy + c] = scale * d;
  }
  rowloss[r] = s;
}
}  // namespace

void mlp_mse(int B, int n_out, const float* y, int ldy, const float* t, int ldt, float* dy, int lddy, double* rowloss,
             cudaStream_t s) {
  ICON_LAUNCH("mlp_mse", (unsigned)((B + 127) / 128), 128, s, mse_kernel, B, n_out, y, ldy, t, ldt, dy, lddy,
              rowloss);
}

}  // namespace icon
