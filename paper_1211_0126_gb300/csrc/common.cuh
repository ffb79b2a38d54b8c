// common.cuh -- device-side building blocks of the TSM library (sm_103a).
//
// Complex arithmetic, even/odd lattice geometry, storage formats of spinors
// and links in FP64 / FP32 / FP16 / BF16, the Philox4x32-10 noise generator,
// and deterministic two-stage FP64 reductions with a device-resident solver
// state.  Everything here is written for this library; nothing is shared with
// the CPU oracle.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace tsm {

// ---------------------------------------------------------------- complex
template <class R>
struct cx {
  R re, im;
};

template <class R> __host__ __device__ __forceinline__ cx<R> mkc(R a, R b) { return cx<R>{a, b}; }
template <class R> __device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <class R> __device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <class R> __device__ __forceinline__ cx<R> operator*(cx<R> a, cx<R> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <class R> __device__ __forceinline__ cx<R> operator*(R s, cx<R> a) { return {s * a.re, s * a.im}; }
template <class R> __device__ __forceinline__ cx<R> cconj(cx<R> a) { return {a.re, -a.im}; }
// conj(a) * b
template <class R> __device__ __forceinline__ cx<R> cjmul(cx<R> a, cx<R> b) {
  return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
template <class R> __device__ __forceinline__ cx<R> times_i(cx<R> a) { return {-a.im, a.re}; }
template <class R> __device__ __forceinline__ R norm2(cx<R> a) { return a.re * a.re + a.im * a.im; }

// ---------------------------------------------------------------- geometry
// Full lattice site index i = x + Lx*(y + Ly*(z + Lz*t)); half-lattice index
// of a site of either parity = i / 2 (Lx even), so each parity is a dense
// array of V/2 sites ordered like the full lattice.
struct Geom {
  int L[4];     // Lx, Ly, Lz, T
  int V, Vh;    // volume, half volume
  int Lxh;      // Lx / 2
  int apbc;     // 1: antiperiodic in t
  // division of a half-site index by Lxh, Ly and Lz as a multiply-high:
  // n / d = umulhi(n, floor(2^32 / d) + 1) exactly whenever n * d < 2^32
  // (n = q d + r: the product's error term n e / 2^32, e <= d, stays below
  // d - r >= 1).  m = 0 marks d = 1.  fastdiv = 0 (Vh * max(L) >= 2^32)
  // falls back to the hardware-free integer division.
  uint32_t mxh, my, mz;
  int fastdiv;
};

inline uint32_t div_magic(int d) { return d <= 1 ? 0u : (uint32_t)((1ull << 32) / (unsigned)d + 1ull); }

// geometry of an Lx x Ly x Lz x T lattice (Lx even)
inline Geom make_geom(const int L[4], int apbc) {
  Geom g{};
  for (int k = 0; k < 4; ++k) g.L[k] = L[k];
  const long long V = (long long)L[0] * L[1] * L[2] * L[3];
  g.V = (int)V;
  g.Vh = (int)(V / 2);
  g.Lxh = L[0] / 2;
  g.apbc = apbc ? 1 : 0;
  g.mxh = div_magic(g.Lxh);
  g.my = div_magic(L[1]);
  g.mz = div_magic(L[2]);
  int lmax = g.Lxh;
  if (L[1] > lmax) lmax = L[1];
  if (L[2] > lmax) lmax = L[2];
  g.fastdiv = (unsigned long long)g.Vh * (unsigned long long)lmax < (1ull << 32) ? 1 : 0;
  return g;
}

__device__ __forceinline__ uint32_t geom_div(const Geom& g, uint32_t n, uint32_t d, uint32_t m) {
  if (g.fastdiv) return m ? __umulhi(n, m) : n;
  return n / d;
}

__device__ __forceinline__ void site_coords(const Geom& g, int parity, int ih, int c[4]) {
  const uint32_t n = (uint32_t)ih;
  const uint32_t r1 = geom_div(g, n, (uint32_t)g.Lxh, g.mxh);
  const int xh = (int)(n - r1 * (uint32_t)g.Lxh);
  const uint32_t r2 = geom_div(g, r1, (uint32_t)g.L[1], g.my);
  const int y = (int)(r1 - r2 * (uint32_t)g.L[1]);
  const uint32_t t = geom_div(g, r2, (uint32_t)g.L[2], g.mz);
  const int z = (int)(r2 - t * (uint32_t)g.L[2]);
  c[0] = 2 * xh + ((parity + y + z + (int)t) & 1);
  c[1] = y;
  c[2] = z;
  c[3] = (int)t;
}

__device__ __forceinline__ int half_index(const Geom& g, int x, int y, int z, int t) {
  return (((t * g.L[2] + z) * g.L[1] + y) * g.L[0] + x) >> 1;
}

// ---------------------------------------------------------------- storage
// A spinor field of one parity is SN "chunks" of Vh elements each (chunk c of
// site i at base[c * stride + i]), so that every load of a warp is coalesced.
// A link field of one parity is 4 directions x LN chunks.  FP32 and 16-bit
// links store rows 0 and 1 only (12 reals), row 2 = conj(row0 x row1) is
// rebuilt in registers; FP64 links store all 18 reals (on GB300 the FP64 pipe,
// not memory, bounds the FP64 stencil, so the rebuild would cost more than the
// extra bytes).
struct F64 {
  using real = double;
  using schunk = double2;   // 1 complex
  using lchunk = double2;
  static constexpr int SN = 12, LN = 9;
  static constexpr bool full_links = true;
  static constexpr int id = 0;
};
struct F32 {
  using real = float;
  using schunk = float4;    // 2 complex
  using lchunk = float4;
  static constexpr int SN = 6, LN = 3;
  static constexpr bool full_links = false;
  static constexpr int id = 1;
};
struct BF16 {
  using real = float;
  using schunk = uint4;     // 4 complex as 8 bf16
  using lchunk = uint2;     // 2 complex as 4 bf16
  static constexpr int SN = 3, LN = 3;
  static constexpr bool full_links = false;
  static constexpr int id = 2;
};
struct F16 {
  using real = float;
  using schunk = uint4;     // 4 complex as 8 fp16
  using lchunk = uint2;     // 2 complex as 4 fp16
  static constexpr int SN = 3, LN = 3;
  static constexpr bool full_links = false;
  static constexpr int id = 3;
};

template <class S> struct Pack16;
template <> struct Pack16<F16> {
  __device__ static __forceinline__ cx<float> unpack(uint32_t w) {
    __half2 h = *reinterpret_cast<const __half2*>(&w);
    float2 f = __half22float2(h);
    return {f.x, f.y};
  }
  __device__ static __forceinline__ uint32_t pack(cx<float> v) {
    __half2 h = __floats2half2_rn(v.re, v.im);
    return *reinterpret_cast<const uint32_t*>(&h);
  }
};
template <> struct Pack16<BF16> {
  __device__ static __forceinline__ cx<float> unpack(uint32_t w) {
    __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162*>(&w);
    float2 f = __bfloat1622float2(h);
    return {f.x, f.y};
  }
  __device__ static __forceinline__ uint32_t pack(cx<float> v) {
    __nv_bfloat162 h = __floats2bfloat162_rn(v.re, v.im);
    return *reinterpret_cast<const uint32_t*>(&h);
  }
};

// load / store of the 12 complex components v[3*spin + colour]
template <class S>
__device__ __forceinline__ void load_spinor(const typename S::schunk* __restrict__ b, int stride, int i,
                                            cx<typename S::real> v[12]) {
  if constexpr (S::id == 0) {
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      double2 d = b[c * stride + i];
      v[c] = {d.x, d.y};
    }
  } else if constexpr (S::id == 1) {
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      float4 f = b[c * stride + i];
      v[2 * c] = {f.x, f.y};
      v[2 * c + 1] = {f.z, f.w};
    }
  } else {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      uint4 u = b[c * stride + i];
      v[4 * c + 0] = Pack16<S>::unpack(u.x);
      v[4 * c + 1] = Pack16<S>::unpack(u.y);
      v[4 * c + 2] = Pack16<S>::unpack(u.z);
      v[4 * c + 3] = Pack16<S>::unpack(u.w);
    }
  }
}

template <class S>
__device__ __forceinline__ void store_spinor(typename S::schunk* __restrict__ b, int stride, int i,
                                             const cx<typename S::real> v[12]) {
  if constexpr (S::id == 0) {
#pragma unroll
    for (int c = 0; c < 12; ++c) b[c * stride + i] = make_double2(v[c].re, v[c].im);
  } else if constexpr (S::id == 1) {
#pragma unroll
    for (int c = 0; c < 6; ++c)
      b[c * stride + i] = make_float4(v[2 * c].re, v[2 * c].im, v[2 * c + 1].re, v[2 * c + 1].im);
  } else {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      uint4 u;
      u.x = Pack16<S>::pack(v[4 * c + 0]);
      u.y = Pack16<S>::pack(v[4 * c + 1]);
      u.z = Pack16<S>::pack(v[4 * c + 2]);
      u.w = Pack16<S>::pack(v[4 * c + 3]);
      b[c * stride + i] = u;
    }
  }
}

// rows of link (dir, site i): r[0..2] = row 0, r[3..5] = row 1 (and r[6..8] =
// row 2 for full-link storage)
template <class S>
__device__ __forceinline__ void load_link(const typename S::lchunk* __restrict__ b, int stride, int dir, int i,
                                          cx<typename S::real> r[9]) {
  const typename S::lchunk* p = b + dir * S::LN * stride + i;
  if constexpr (S::id == 0) {
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      double2 d = p[c * stride];
      r[c] = {d.x, d.y};
    }
  } else if constexpr (S::id == 1) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float4 f = p[c * stride];
      r[2 * c] = {f.x, f.y};
      r[2 * c + 1] = {f.z, f.w};
    }
  } else {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      uint2 u = p[c * stride];
      r[2 * c] = Pack16<S>::unpack(u.x);
      r[2 * c + 1] = Pack16<S>::unpack(u.y);
    }
  }
}

template <class S>
__device__ __forceinline__ void store_link(typename S::lchunk* __restrict__ b, int stride, int dir, int i,
                                           const cx<typename S::real> r[9]) {
  typename S::lchunk* p = b + dir * S::LN * stride + i;
  if constexpr (S::id == 0) {
#pragma unroll
    for (int c = 0; c < 9; ++c) p[c * stride] = make_double2(r[c].re, r[c].im);
  } else if constexpr (S::id == 1) {
#pragma unroll
    for (int c = 0; c < 3; ++c) p[c * stride] = make_float4(r[2 * c].re, r[2 * c].im, r[2 * c + 1].re, r[2 * c + 1].im);
  } else {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      uint2 u;
      u.x = Pack16<S>::pack(r[2 * c]);
      u.y = Pack16<S>::pack(r[2 * c + 1]);
      p[c * stride] = u;
    }
  }
}

// third row of an SU(3) matrix from its first two: row2 = conj(row0 x row1)
template <class R>
__device__ __forceinline__ void third_row(const cx<R> r[6], cx<R> w[3]) {
  w[0] = cconj(r[1] * r[5] - r[2] * r[4]);
  w[1] = cconj(r[2] * r[3] - r[0] * r[5]);
  w[2] = cconj(r[0] * r[4] - r[1] * r[3]);
}

// ---------------------------------------------------------------- twist
// Site-local factors diagonal in the chiral basis: spins 0,1 times f[0],
// spins 2,3 times f[1].  A(mu) = 1 + 2 i kappa mu gamma_5 -> f = (1 + 2i k mu, 1 - 2i k mu).
struct Twist {
  double re[2], im[2];
};

// the same factors rounded once on the host for the FP32-arithmetic kernels
// (a double-to-float conversion per thread runs on GB300's narrow FP64 pipe)
struct TwistF {
  float re[2], im[2];
};

inline TwistF to_float(const Twist& t) {
  return TwistF{{(float)t.re[0], (float)t.re[1]}, {(float)t.im[0], (float)t.im[1]}};
}

template <class R>
__device__ __forceinline__ void apply_twist(const TwistF& f, cx<R> v[12]) {
  const cx<R> a = {f.re[0], f.im[0]}, b = {f.re[1], f.im[1]};
#pragma unroll
  for (int k = 0; k < 6; ++k) v[k] = a * v[k];
#pragma unroll
  for (int k = 6; k < 12; ++k) v[k] = b * v[k];
}

template <class R>
__device__ __forceinline__ void apply_twist(const Twist& f, cx<R> v[12]) {
  cx<R> a = {(R)f.re[0], (R)f.im[0]};
  cx<R> b = {(R)f.re[1], (R)f.im[1]};
#pragma unroll
  for (int k = 0; k < 6; ++k) v[k] = a * v[k];
#pragma unroll
  for (int k = 6; k < 12; ++k) v[k] = b * v[k];
}

// ---------------------------------------------------------------- Philox4x32-10
// Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3"
// (SC'11): ten rounds of two 32x32->64 multiplies with a Weyl-sequence key.
__device__ __forceinline__ uint32_t philox_word0(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                 uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c0;
}

struct NoiseSpec {
  uint32_t k0, k1;   // seed low / high word
  int kind;          // 4 = Z4, 2 = Z2
  double amp;        // 1/sqrt(2) for Z4 (host-computed), 1 for Z2
  float famp;        // amp rounded once on the host (FP32 kernels: no conversion on the FP64 pipe)
};

// eta_source at full-lattice site `lex`, component a = 3*spin + colour
template <class R>
__device__ __forceinline__ void noise_site(const NoiseSpec& n, uint32_t lex, uint32_t source, cx<R> v[12]) {
  const uint32_t w = philox_word0(lex, source, 0u, 0u, n.k0, n.k1);
  const R amp = sizeof(R) == 4 ? (R)n.famp : (R)n.amp;
#pragma unroll
  for (int a = 0; a < 12; ++a) {
    const R re = ((w >> (2 * a)) & 1u) ? -amp : amp;
    const R im = (n.kind == 4) ? (((w >> (2 * a + 1)) & 1u) ? -amp : amp) : (R)0;
    v[a] = {re, im};
  }
}

// ---------------------------------------------------------------- solver state
// One per right-hand side, in device memory.  Reductions finish in the last
// block of the reducing kernel, which updates this state; every CG kernel
// returns at once when `done` is set, so iterates freeze exactly at the
// iteration that met the stopping rule even if more iterations are queued.
struct CGState {
  double rr;        // <r, r> of the current iterate
  double rr0;       // <Dhat^dag bhat, Dhat^dag bhat>
  double pAp;       // <Dhat p, Dhat p>
  double alpha, beta;
  float alpha_f, beta_f;   // alpha, beta rounded once for the FP32 kernels
  double tol;       // rel_tol
  double aux;       // scratch result (norms of helper reductions)
  double rr_ref;    // <r, r> at the last reliable update
  double delta2;    // reliable update when rr < delta2 * rr_ref
  int iter, max_iter;
  int done;         // 1: stopping rule met (or cap reached / error)
  int status;       // 0 ok, TSM_ERR_NONFINITE on NaN/Inf
  int rel;          // 1: FP64 reliable updates (FP32 iterations)
  int need_rel;     // 1: a reliable update is due before the next iteration
  int final_check;  // 1: the iterated residual met the rule; the update decides
};

enum PostOp {
  POST_NONE = 0,    // write the sum to st->aux
  POST_INIT = 1,    // rr = rr0 = rr_ref = sum, iter = 0, done per stopping rule
  POST_ALPHA = 2,   // pAp = sum, alpha = rr / pAp
  POST_RR = 3,      // rr' = sum: beta = rr'/rr, rr = rr', iter++, stopping rule
  POST_SETRR = 4    // rr = rr_ref = sum (true residual of a reliable update)
};

// stopping rule of the iterated residual: ||r|| < tol ||r0|| (NaN counts as met)
__device__ __forceinline__ bool rule_met(const CGState* st, double rr) {
  return !(sqrt(rr) >= st->tol * sqrt(st->rr0));
}

__device__ __forceinline__ void post_action(CGState* st, int op, double sum) {
  if (st == nullptr) return;
  const bool finite = isfinite(sum);
  switch (op) {
    case POST_NONE:
      st->aux = sum;
      break;
    case POST_INIT:
      st->rr = sum;
      st->rr0 = sum;
      st->rr_ref = sum;
      st->iter = 0;
      st->need_rel = 0;
      st->final_check = 0;
      st->status = finite ? 0 : -5;
      st->done = (!finite || sum == 0.0 || st->max_iter <= 0 || !(sqrt(sum) >= st->tol * sqrt(sum))) ? 1 : 0;
      break;
    case POST_ALPHA:
      st->pAp = sum;
      st->alpha = st->rr / sum;
      st->alpha_f = (float)st->alpha;
      if (!finite || !isfinite(st->alpha)) {
        st->status = -5;
        st->done = 1;
      }
      break;
    case POST_RR: {
      st->beta = sum / st->rr;
      st->beta_f = (float)st->beta;
      st->rr = sum;
      st->iter += 1;
      if (!finite) {
        st->status = -5;
        st->done = 1;
      } else if (st->iter >= st->max_iter || rule_met(st, sum)) {
        // with reliable updates the FP64 residual of the update decides
        if (st->rel) {
          st->need_rel = 1;
          st->final_check = 1;
        } else {
          st->done = 1;
        }
      } else if (st->rel && sum < st->delta2 * st->rr_ref) {
        st->need_rel = 1;
      }
      break;
    }
    case POST_SETRR:
      st->rr = sum;
      st->rr_ref = sum;
      if (!finite) {
        st->status = -5;
        st->done = 1;
      }
      break;
  }
}

// ---------------------------------------------------------------- reductions
// Two-stage deterministic sum per right-hand side: the blocks of one RHS are
// blockIdx.y = 0 .. gridDim.y-1 (blockIdx.x selects the RHS); every block
// writes its partial to partials[rhs * stride + block]; the last block of
// that RHS to finish (atomic ticket) adds the partials in block order and
// applies the post action.  The ticket counter is reset by that block so the
// slot can be reused by the next launch.  The sum of one RHS therefore does
// not depend on which other right-hand sides share the launch.
struct RedSlot {
  double* partials;       // [rhs][stride]
  unsigned int* counter;  // [rhs]
  int stride;
};

// fixed-order block sum: the warp stage in the value's own type (an FP32
// partial stays FP32 across the 32 lanes, off GB300's narrow FP64 pipe), the
// warps' sums in FP64
template <int NT, class V>
__device__ __forceinline__ double block_sum(V v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sh[warp] = (double)v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) s += sh[w];
  }
  __syncthreads();
  return s;  // valid in thread 0
}

// p[first] + p[first + step] + ... (indices below n) added in increasing
// index order, with eight loads in flight at a time: the same sum, bit for
// bit, as the plain loop, without one L2 round trip per term
__device__ __forceinline__ double strided_sum_ordered(const double* p, int first, int n, int step) {
  double acc = 0.0;
  int b = first;
  for (; b + 7 * step < n; b += 8 * step) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = __ldcg(p + b + u * step);
#pragma unroll
    for (int u = 0; u < 8; ++u) acc += v[u];
  }
  for (; b < n; b += step) acc += __ldcg(p + b);
  return acc;
}

// Called by all threads of every block of right-hand side `rhs`.  Returns
// true in the last block of that RHS, in which thread 0 holds its total.
template <int NT, class V>
__device__ __forceinline__ bool grid_sum(V v, RedSlot slot, int rhs, double* total) {
  __shared__ double sh[NT / 32];
  __shared__ bool is_last;
  const int nblocks = gridDim.y;
  double* partials = slot.partials + (size_t)rhs * slot.stride;
  unsigned int* counter = slot.counter + rhs;
  double s = block_sum<NT>(v, sh);
  if (threadIdx.x == 0) {
    partials[blockIdx.y] = s;
    __threadfence();
    const unsigned int ticket = atomicAdd(counter, 1u);
    is_last = (ticket == (unsigned int)(nblocks - 1));
  }
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  const double acc = strided_sum_ordered(partials, threadIdx.x, nblocks, NT);
  // fixed-order tree over the threads' strided partial sums
  double tot = block_sum<NT>(acc, sh);
  if (threadIdx.x == 0) {
    *total = tot;
    *counter = 0u;
  }
  return true;
}

// right-hand side handled by this block: blockIdx.x, or the entry of an
// active list (converged right-hand sides are left out of later launches)
__device__ __forceinline__ int rhs_slot(const int* active) {
  return active != nullptr ? active[blockIdx.x] : (int)blockIdx.x;
}

// offset of right-hand side `rhs` in a batch of contiguous fields of storage S
template <class S>
__device__ __forceinline__ size_t rhs_offset(int rhs, int sstride) {
  return (size_t)rhs * S::SN * (size_t)sstride;
}

}  // namespace tsm
