// umma.cuh -- BF16 GEMM on the 5th-generation tensor cores (tcgen05, sm_103a).
//
//   C[M x N] (FP32) = A[M x K] (BF16, row-major) * B[N x K]^T (BF16, row-major)
//
// used by the channel-mixing layers of the learned preconditioner.  One CTA
// (128 threads) computes a 128 x BN tile: the operand tiles are staged in
// shared memory in the canonical K-major layout without swizzle (8-row x
// 16-byte core matrices, K-adjacent cores 128 B apart, 8-row groups
// (K_TILE / 8) * 128 B apart), one elected thread issues tcgen05.mma with the
// accumulator in tensor memory (TMEM), completion is signalled through an
// mbarrier by tcgen05.commit, and the epilogue reads TMEM with tcgen05.ld.
// Every wait is bounded: on timeout the CTA records an error flag, still
// frees its TMEM and returns.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace tsm {

constexpr int UMMA_BM = 128;
constexpr int UMMA_BK = 64;              // K elements per shared-memory stage (4 MMAs of K = 16)
constexpr int UMMA_THREADS = 128;
constexpr long long UMMA_SPIN_LIMIT = 1ll << 26;   // bounded mbarrier wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor: canonical K-major layout without swizzle
// (start address, leading-dimension byte offset = distance of K-adjacent core
// matrices, stride byte offset = distance of adjacent 8-row groups)
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;   // descriptor version for tcgen05
  return d;                 // base offset 0, no swizzle
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N and M encoded as N/8 and M/16
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

// bounded wait for the phase `parity` of an mbarrier; false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (long long it = 0; it < UMMA_SPIN_LIMIT; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// tile of R rows x UMMA_BK columns of a row-major BF16 matrix (leading
// dimension ld, rows >= nrows / columns >= ncols zero-filled) -> canonical
// K-major core-matrix layout in shared memory
template <int R>
__device__ __forceinline__ void stage_tile(const __nv_bfloat16* __restrict__ g, int ld, int row0, int nrows, int k0,
                                           int ncols, uint8_t* s) {
  // R rows x 8 chunks of 16 bytes (8 BF16 each)
  for (int idx = threadIdx.x; idx < R * (UMMA_BK / 8); idx += UMMA_THREADS) {
    const int r = idx / (UMMA_BK / 8), kc = idx % (UMMA_BK / 8);
    const int row = row0 + r, col = k0 + kc * 8;
    uint4 v = make_uint4(0, 0, 0, 0);
    if (row < nrows) {
      if (col + 8 <= ncols) {
        v = *reinterpret_cast<const uint4*>(g + (size_t)row * ld + col);
      } else if (col < ncols) {
        __nv_bfloat16 tmp[8];
        for (int e = 0; e < 8; ++e) tmp[e] = (col + e < ncols) ? g[(size_t)row * ld + col + e] : __float2bfloat16(0.f);
        v = *reinterpret_cast<uint4*>(tmp);
      }
    }
    // core matrix (r / 8, kc): 8 rows x 16 B; K-adjacent cores 128 B apart
    const int off = ((r >> 3) * (UMMA_BK / 8) + kc) * 128 + (r & 7) * 16;
    *reinterpret_cast<uint4*>(s + off) = v;
  }
}

// C = A * B^T  (A: M x K, B: N x K, row-major BF16; C: M x N FP32 row-major,
// leading dimension ldc; beta = 0 overwrites, 1 accumulates into C).
// BN = tile width (multiple of 16, <= 192: the static shared memory holds
// both stages within 48 KB); K need not be a multiple of 64
// (zero-filled) but the rows of A and B must start 16-byte aligned (K % 8 == 0).
//
// Split-K: blockIdx.z covers K range [z * kchunk, (z + 1) * kchunk) and writes
// its partial product to C + z * czstride (reduced afterwards by the caller).
template <int BN>
__global__ void __launch_bounds__(UMMA_THREADS) umma_gemm_kernel(const __nv_bfloat16* __restrict__ A,
                                                                 const __nv_bfloat16* __restrict__ B,
                                                                 float* __restrict__ C, int M, int N, int K,
                                                                 int ldc, int beta, int* __restrict__ error,
                                                                 int lda, int ldb, int kchunk, long long czstride) {
  static_assert(BN % 16 == 0 && BN >= 16 && BN <= 192, "BN must be a multiple of 16 in [16, 192]");
  constexpr int TMEM_COLS = BN <= 32 ? 32 : (BN <= 64 ? 64 : (BN <= 128 ? 128 : 256));
  __shared__ __align__(1024) uint8_t sA[UMMA_BM * UMMA_BK * 2];
  __shared__ __align__(1024) uint8_t sB[BN * UMMA_BK * 2];
  __shared__ __align__(8) uint64_t mma_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int timed_out;
  const int m0 = blockIdx.x * UMMA_BM, n0 = blockIdx.y * BN;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    mbar_init(&mma_bar, 1);
    timed_out = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  constexpr uint32_t idesc = umma_idesc_bf16(UMMA_BM, BN);
  // this CTA's K range (split-K along blockIdx.z)
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(K, kbeg + kchunk);
  const int ktiles = kend > kbeg ? (kend - kbeg + UMMA_BK - 1) / UMMA_BK : 0;
  C += (size_t)blockIdx.z * (size_t)czstride;
  uint32_t phase = 0;
  for (int kt = 0; kt < ktiles; ++kt) {
    stage_tile<UMMA_BM>(A, lda, m0, M, kbeg + kt * UMMA_BK, kend, sA);
    stage_tile<BN>(B, ldb, n0, N, kbeg + kt * UMMA_BK, kend, sB);
    // generic-proxy writes of shared memory -> visible to the tensor core (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
#pragma unroll
      for (int kk = 0; kk < UMMA_BK / 16; ++kk) {
        // K = 16 per MMA = two K-adjacent core matrices (256 B further per step)
        const uint64_t da = umma_desc(a0 + kk * 256, 128, (UMMA_BK / 8) * 128);
        const uint64_t db = umma_desc(b0 + kk * 256, 128, (UMMA_BK / 8) * 128);
        const uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(da), "l"(db), "r"(idesc), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&mma_bar))
                   : "memory");
    }
    // wait until the MMAs of this stage have read shared memory and finished
    if (!mbar_wait(&mma_bar, phase)) timed_out = 1;
    phase ^= 1u;
    __syncthreads();
    if (timed_out) break;
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!timed_out) {
    // epilogue: warp w owns accumulator lanes (rows) 32w .. 32w+31 (an empty
    // split-K range contributes zeros)
    const int row = m0 + warp * 32 + lane;
    for (int c0 = 0; c0 < BN; c0 += 8) {
      uint32_t v[8];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (ktiles == 0) {
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = 0u;
      }
      if (row < M) {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int col = n0 + c0 + e;
          if (col < N) {
            float* dst = C + (size_t)row * ldc + col;
            const float val = __uint_as_float(v[e]);
            *dst = beta ? *dst + val : val;
          }
        }
      }
    }
  }
  if (timed_out) {
    // give MMAs still in flight a second bounded wait before TMEM is released
    mbar_wait(&mma_bar, phase);
    if (threadIdx.x == 0 && error != nullptr) atomicExch(error, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
  }
}

}  // namespace tsm
