// umma.cuh -- BF16 GEMM on the 5th-generation tensor cores (tcgen05, sm_103a).
//
//   C[M x N] (FP32) = A[M x K] (BF16, row-major) * B[N x K]^T (BF16, row-major)
//
// used by the channel-mixing layers of the learned preconditioner.  One CTA
// (128 threads) computes a 128 x BN tile of C over its K range through a
// 3- or 4-deep ring of shared-memory stages: all threads copy operand
// tiles with cp.async (16 bytes per copy, zero fill outside the matrices)
// into the canonical K-major layout without swizzle (8-row x 16-byte core
// matrices, K-adjacent cores 128 B apart, 8-row groups (UMMA_BK / 8) * 128 B
// apart) while one thread issues tcgen05.mma on the stage that has landed,
// with the accumulator in tensor memory (TMEM).  tcgen05.commit arrives on the
// stage's mbarrier when its MMAs are done, which frees the stage for the copy
// UMMA_STAGES - 1 tiles ahead.  The epilogue reads TMEM with tcgen05.ld.
// Every wait is bounded: on timeout the CTA records an error flag, waits
// (bounded) for its copies and MMAs in flight, frees its TMEM and returns.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace tsm {

constexpr int UMMA_BM = 128;
constexpr int UMMA_BK = 64;              // K elements per shared-memory stage (4 MMAs of K = 16)
constexpr int UMMA_THREADS = 128;
constexpr int UMMA_A_BYTES = UMMA_BM * UMMA_BK * 2;
// ring depth: 4 stages for narrow tiles, 3 for BN >= 64 so that two CTAs fit
// in one SM's shared memory (one CTA's epilogue overlaps the other's loads)
template <int BN> __host__ __device__ constexpr int umma_stages() { return BN >= 64 ? 3 : 4; }
template <int BN> __host__ __device__ constexpr int umma_stage_bytes() { return UMMA_A_BYTES + BN * UMMA_BK * 2; }
template <int BN> __host__ __device__ constexpr int umma_smem_bytes() {
  return umma_stages<BN>() * umma_stage_bytes<BN>() + 1024;
}
constexpr long long UMMA_SPIN_LIMIT = 1ll << 26;   // bounded mbarrier wait
// stage-wait limit of a launch with withheld operand copies (fault injection
// for tests of the timeout path): the wait is on a barrier nothing arrives on
constexpr long long UMMA_INJECT_LIMIT = 4096;

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
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit = UMMA_SPIN_LIMIT) {
  const uint32_t a = smem_u32(bar);
  for (long long it = 0; it < limit; ++it) {
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

// cp.async of one R-row x UMMA_BK-column tile of a row-major BF16 matrix
// (leading dimension ld; rows >= nrows and columns >= ncols are zero-filled;
// ncols and ld multiples of 8) into the canonical K-major core-matrix layout
template <int R>
__device__ __forceinline__ void copy_tile_async(const __nv_bfloat16* __restrict__ g, int ld, int row0, int nrows,
                                                int k0, int ncols, uint32_t s) {
#pragma unroll 2
  for (int idx = threadIdx.x; idx < R * (UMMA_BK / 8); idx += UMMA_THREADS) {
    const int r = idx / (UMMA_BK / 8), kc = idx % (UMMA_BK / 8);
    const int row = row0 + r, col = k0 + kc * 8;
    const bool in = row < nrows && col < ncols;
    const __nv_bfloat16* src = in ? g + (size_t)row * ld + col : g;   // valid address, nothing read when !in
    const uint32_t dst = s + ((r >> 3) * (UMMA_BK / 8) + kc) * 128 + (r & 7) * 16;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(in ? 16 : 0)
                 : "memory");
  }
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// C = A * B^T  (A: M x K, B: N x K, row-major BF16; C: M x N FP32 row-major,
// leading dimension ldc; beta = 0 overwrites, 1 accumulates into C).
// BN = tile width (multiple of 16 in [16, 256]); K, lda, ldb multiples of 8.
// Split-K: blockIdx.z covers K range [z * kchunk, (z + 1) * kchunk) (kchunk a
// multiple of UMMA_BK) and writes its partial product to C + z * czstride.
// Dynamic shared memory: umma_smem_bytes<BN>().
template <int BN>
__global__ void __launch_bounds__(UMMA_THREADS) umma_gemm_kernel(const __nv_bfloat16* __restrict__ A,
                                                                 const __nv_bfloat16* __restrict__ B,
                                                                 float* __restrict__ C, int M, int N, int K,
                                                                 int ldc, int beta, int* __restrict__ error,
                                                                 int lda, int ldb, int kchunk, long long czstride) {
  static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "BN must be a multiple of 16 in [16, 256]");
  constexpr int TMEM_COLS = BN <= 32 ? 32 : (BN <= 64 ? 64 : (BN <= 128 ? 128 : 256));
  constexpr int SB = umma_stage_bytes<BN>();
  constexpr int UMMA_STAGES = umma_stages<BN>();
  extern __shared__ uint8_t umma_dyn[];
  __shared__ __align__(8) uint64_t bar[UMMA_STAGES];
  __shared__ uint32_t tmem_slot;
  __shared__ int timed_out;
  // 1024-byte aligned ring of stages
  const uint32_t ring = (smem_u32(umma_dyn) + 1023u) & ~1023u;
  const int m0 = blockIdx.x * UMMA_BM, n0 = blockIdx.y * BN;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int s = 0; s < UMMA_STAGES; ++s) mbar_init(&bar[s], 1);
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
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(K, kbeg + kchunk);
  const int ktiles = kend > kbeg ? (kend - kbeg + UMMA_BK - 1) / UMMA_BK : 0;
  C += (size_t)blockIdx.z * (size_t)czstride;
  int last = -1;   // last tile whose MMAs were committed
  auto load = [&](int kt, int s) {
    const uint32_t sa = ring + s * SB;
    copy_tile_async<UMMA_BM>(A, lda, m0, M, kbeg + kt * UMMA_BK, kend, sa);
    copy_tile_async<BN>(B, ldb, n0, N, kbeg + kt * UMMA_BK, kend, sa + UMMA_A_BYTES);
  };
  // prologue: tiles 0 .. STAGES-2 in flight (one commit group per tile, empty groups keep the count)
#pragma unroll
  for (int s = 0; s < UMMA_STAGES - 1; ++s) {
    if (s < ktiles) load(s, s);
    cp_async_commit();
  }
  for (int kt = 0; kt < ktiles; ++kt) {
    const int s = kt % UMMA_STAGES;
    cp_async_wait<UMMA_STAGES - 2>();   // this thread's copies of tile kt have landed
    // generic-proxy writes of shared memory -> visible to the tensor core (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = ring + s * SB, b0 = a0 + UMMA_A_BYTES;
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
                       smem_u32(&bar[s]))
                   : "memory");
    }
    last = kt;
    // refill the stage of tile kt-1 with tile kt+STAGES-1 once tile kt-1's MMAs are done
    const int nk = kt + UMMA_STAGES - 1;
    if (nk < ktiles) {
      const int ps = nk % UMMA_STAGES;
      if (kt >= 1 && !mbar_wait(&bar[ps], (uint32_t)(((kt - 1) / UMMA_STAGES) & 1))) timed_out = 1;
      __syncthreads();
      if (timed_out) break;
      load(nk, ps);
    }
    cp_async_commit();
  }
  // all MMAs done: the commit of the last tile covers every earlier MMA
  if (last >= 0 && !timed_out) {
    if (!mbar_wait(&bar[last % UMMA_STAGES], (uint32_t)((last / UMMA_STAGES) & 1))) timed_out = 1;
  }
  cp_async_wait<0>();
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!timed_out) {
    // epilogue: warp w owns accumulator lanes (rows) 32w .. 32w+31 (an empty
    // split-K range contributes zeros)
    const int row = m0 + warp * 32 + lane;
    const bool vec = (ldc % 4) == 0 && (reinterpret_cast<uintptr_t>(C) & 15) == 0;
    for (int c0 = 0; c0 < BN; c0 += 8) {
      uint32_t v[8];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      float f[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) f[e] = ktiles == 0 ? 0.f : __uint_as_float(v[e]);
      const int col = n0 + c0;
      if (row < M && col < N) {
        float* dst = C + (size_t)row * ldc + col;
        if (vec && col + 8 <= N) {
          float4 lo = make_float4(f[0], f[1], f[2], f[3]), hi = make_float4(f[4], f[5], f[6], f[7]);
          if (beta) {
            const float4 a = *reinterpret_cast<const float4*>(dst), b = *reinterpret_cast<const float4*>(dst + 4);
            lo = make_float4(lo.x + a.x, lo.y + a.y, lo.z + a.z, lo.w + a.w);
            hi = make_float4(hi.x + b.x, hi.y + b.y, hi.z + b.z, hi.w + b.w);
          }
          *reinterpret_cast<float4*>(dst) = lo;
          *reinterpret_cast<float4*>(dst + 4) = hi;
        } else {
#pragma unroll
          for (int e = 0; e < 8; ++e)
            if (col + e < N) dst[e] = beta ? dst[e] + f[e] : f[e];
        }
      }
    }
  } else {
    // give MMAs still in flight a second bounded wait before TMEM is released
    if (last >= 0) mbar_wait(&bar[last % UMMA_STAGES], (uint32_t)((last / UMMA_STAGES) & 1));
    if (threadIdx.x == 0 && error != nullptr) atomicExch(error, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
  }
}

}  // namespace tsm

// ---------------------------------------------------------------- TMA-fed variant
// The same product with the operand tiles brought in by the tensor memory
// accelerator: thread 0 issues, per stage, one box of 64 columns x 128 rows
// of A and one of 64 columns x BN rows of B (cp.async.bulk.tensor with
// 128-byte swizzle, zero fill outside the matrices) onto an mbarrier with an
// expected byte count.  Rows land 128 B apart with their 16-byte chunks
// XOR-permuted within each 1024-byte group of 8 rows -- the canonical K-major
// SWIZZLE_128B layout of the MMA descriptors (8-row groups 1024 B apart; the
// K = 16 slices of a stage are 32 B apart inside the swizzle atom).  Thread 32
// waits for a stage, issues its four MMAs and lets tcgen05.commit release the
// stage to the producer; a last commit signals the accumulator to the
// epilogue.  No thread-wide barrier inside the K loop.  Every wait is bounded;
// on timeout the CTA records the error, waits (bounded) for the copies it
// issued and for its MMAs, frees TMEM and returns.  withhold = 1 (fault
// injection for tests) issues no copies and gives the stage waits a limit of
// UMMA_INJECT_LIMIT polls: the MMA thread's first wait, on a stage nothing
// fills, runs out; no copy and no MMA is in flight, so the done and clean-up
// waits (full limit) end at once.
namespace tsm {

constexpr int UMMA_TMA_BOX_K = UMMA_BK;   // columns per TMA box: 64 BF16 = one 128-byte swizzle span

// shared-memory matrix descriptor, canonical K-major layout with 128-byte
// swizzle: 8-row groups 1024 B apart (SBO), leading offset unused (1)
__device__ __forceinline__ uint64_t umma_desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;   // descriptor version for tcgen05
  d |= (uint64_t)2 << 61;   // swizzle mode: 128 B
  return d;
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void* tmap, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(tmap), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

template <int BN> __host__ __device__ constexpr int umma_tma_stages() { return BN >= 64 ? 3 : 4; }
template <int BN> __host__ __device__ constexpr int umma_tma_smem_bytes() {
  return umma_tma_stages<BN>() * umma_stage_bytes<BN>() + 1024;
}

template <int BN>
__global__ void __launch_bounds__(UMMA_THREADS) umma_tma_gemm_kernel(const __grid_constant__ CUtensorMap ta,
                                                                     const __grid_constant__ CUtensorMap tb,
                                                                     float* __restrict__ C, int M, int N, int K,
                                                                     int ldc, int beta, int* __restrict__ error,
                                                                     int kchunk, long long czstride, int withhold) {
  static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "BN must be a multiple of 16 in [16, 256]");
  constexpr int TMEM_COLS = BN <= 32 ? 32 : (BN <= 64 ? 64 : (BN <= 128 ? 128 : 256));
  constexpr int ST = umma_tma_stages<BN>();
  constexpr int SB = umma_stage_bytes<BN>();
  constexpr uint32_t STAGE_TX = (uint32_t)(UMMA_BM + BN) * UMMA_BK * 2;
  extern __shared__ uint8_t umma_dyn[];
  __shared__ __align__(8) uint64_t full[ST], empty[ST], done;
  __shared__ uint32_t tmem_slot;
  __shared__ int timed_out, issued, consumed;
  const uint32_t ring = (smem_u32(umma_dyn) + 1023u) & ~1023u;
  const int m0 = blockIdx.x * UMMA_BM, n0 = blockIdx.y * BN;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int s = 0; s < ST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&done, 1);
    timed_out = 0;
    issued = 0;
    consumed = 0;
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
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(K, kbeg + kchunk);
  const int ktiles = kend > kbeg ? (kend - kbeg + UMMA_BK - 1) / UMMA_BK : 0;
  C += (size_t)blockIdx.z * (size_t)czstride;
  const long long stage_limit = withhold ? UMMA_INJECT_LIMIT : UMMA_SPIN_LIMIT;
  if (threadIdx.x == 0) {
    // producer
    for (int kt = 0; kt < ktiles && !withhold; ++kt) {
      const int s = kt % ST;
      if (kt >= ST && !mbar_wait(&empty[s], (uint32_t)(((kt / ST) - 1) & 1), stage_limit)) {
        atomicExch(&timed_out, 1);
        break;
      }
      if (*reinterpret_cast<volatile int*>(&timed_out)) break;
      mbar_expect_tx(&full[s], STAGE_TX);
      const uint32_t sa = ring + s * SB, sb = sa + UMMA_A_BYTES;
      const int k0 = kbeg + kt * UMMA_BK;
      tma_load_2d(sa, &ta, k0, m0, &full[s]);
      tma_load_2d(sb, &tb, k0, n0, &full[s]);
      *reinterpret_cast<volatile int*>(&issued) = kt + 1;
    }
  } else if (threadIdx.x == 32) {
    // MMA issuer
    for (int kt = 0; kt < ktiles; ++kt) {
      const int s = kt % ST;
      if (!mbar_wait(&full[s], (uint32_t)((kt / ST) & 1), stage_limit)) {
        atomicExch(&timed_out, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = ring + s * SB, b0 = a0 + UMMA_A_BYTES;
#pragma unroll
      for (int kk = 0; kk < UMMA_BK / 16; ++kk) {
        // K = 16 per MMA = 32 bytes further inside the 128-byte swizzle span
        const uint64_t da = umma_desc_sw128(a0 + kk * 32);
        const uint64_t db = umma_desc_sw128(b0 + kk * 32);
        const uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(da), "l"(db), "r"(idesc), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&empty[s]))
                   : "memory");
      *reinterpret_cast<volatile int*>(&consumed) = kt + 1;
    }
    // the accumulator is complete when every MMA issued so far is
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(&done))
                 : "memory");
  }
  __syncthreads();
  if (!mbar_wait(&done, 0)) atomicExch(&timed_out, 1);
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!timed_out) {
    const int row = m0 + warp * 32 + lane;
    const bool vec = (ldc % 4) == 0 && (reinterpret_cast<uintptr_t>(C) & 15) == 0;
    for (int c0 = 0; c0 < BN; c0 += 8) {
      uint32_t v[8];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      float f[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) f[e] = ktiles == 0 ? 0.f : __uint_as_float(v[e]);
      const int col = n0 + c0;
      if (row < M && col < N) {
        float* dst = C + (size_t)row * ldc + col;
        if (vec && col + 8 <= N) {
          float4 lo = make_float4(f[0], f[1], f[2], f[3]), hi = make_float4(f[4], f[5], f[6], f[7]);
          if (beta) {
            const float4 a = *reinterpret_cast<const float4*>(dst), b = *reinterpret_cast<const float4*>(dst + 4);
            lo = make_float4(lo.x + a.x, lo.y + a.y, lo.z + a.z, lo.w + a.w);
            hi = make_float4(hi.x + b.x, hi.y + b.y, hi.z + b.z, hi.w + b.w);
          }
          *reinterpret_cast<float4*>(dst) = lo;
          *reinterpret_cast<float4*>(dst + 4) = hi;
        } else {
#pragma unroll
          for (int e = 0; e < 8; ++e)
            if (col + e < N) dst[e] = beta ? dst[e] + f[e] : f[e];
        }
      }
    }
  } else if (threadIdx.x == 0) {
    // let the copies already issued land before the shared memory goes away
    const int n_issued = *reinterpret_cast<volatile int*>(&issued);
    const int n_used = *reinterpret_cast<volatile int*>(&consumed);
    for (int kt = n_used; kt < n_issued; ++kt) mbar_wait(&full[kt % ST], (uint32_t)((kt / ST) & 1));
    if (error != nullptr) atomicExch(error, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
  }
}

}  // namespace tsm
