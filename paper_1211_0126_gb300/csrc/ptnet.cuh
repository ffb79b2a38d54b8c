// ptnet.cuh -- kernels of the parallel-transport network (learned LP preconditioner).
//
// A layer maps C_in complex channels (each a spinor field) to C_out:
//   y_{c'}(x)_{s' a} = sum_{p=0..8} sum_{c,s} W[(c',s'),(p,c,s)] (T_p psi_c)(x)_{s a}
// with T_0 = 1, T_{2mu+1} psi(x) = U_mu(x) psi(x+mu), T_{2mu+2} psi(x) =
// U_mu(x-mu)^dag psi(x-mu) (fermion boundary sign across t = T-1 <-> 0).
// It runs as: gather (transport, BF16 output) -> tensor-core GEMM
// Y = Z * B^T with the real block form B = [[Wr, -Wi], [Wi, Wr]].
//
// Activation rows m = 3 * site + colour (lexicographic full-lattice site);
// an activation with C channels has 8C FP32 columns: real parts
// (c * 4 + s) in [0, 4C), imaginary parts at 4C + (c * 4 + s).  The gathered
// matrix Z has 72 C BF16 columns: for each (path p, channel c), j = p * C + c,
// the 16-byte group 8 j .. 8 j + 7 holds the real parts of spins 0..3 and
// then their imaginary parts (one core-matrix row of the tensor-core layout).
// The block weight matrix B [8 C_out][72 C_in] matches: row n < 4 C_out gives
// the real part of output component n, row 4 C_out + n its imaginary part.
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace tsm {

constexpr int NET_NT = 256;
constexpr int PT_PATHS = 9;

struct NetGeom {
  Geom g;
  const float4* links;   // FP32 two-row links [2 parities][4 dirs][3 chunks][lstride]
  int lstride;
};

__device__ __forceinline__ void lex_coords(const Geom& g, int lex, int c[4]) {
  int r = lex;
  c[0] = r % g.L[0];
  r /= g.L[0];
  c[1] = r % g.L[1];
  r /= g.L[1];
  c[2] = r % g.L[2];
  c[3] = r / g.L[2];
}

__device__ __forceinline__ int lex_of(const Geom& g, const int c[4]) {
  return ((c[3] * g.L[2] + c[2]) * g.L[1] + c[1]) * g.L[0] + c[0];
}

// one channel's 4 x 3 complex components at site `lex` of an activation
__device__ __forceinline__ void load_channel(const float* __restrict__ X, int C, int lex, int ch, cx<float> v[4][3]) {
  const int w = 8 * C;
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    const float* row = X + (size_t)(3 * lex + b) * w;
    const float4 re = *reinterpret_cast<const float4*>(row + ch * 4);
    const float4 im = *reinterpret_cast<const float4*>(row + 4 * C + ch * 4);
    v[0][b] = {re.x, im.x};
    v[1][b] = {re.y, im.y};
    v[2][b] = {re.z, im.z};
    v[3][b] = {re.w, im.w};
  }
}

// neighbour of site (x0..x3) along path p = 1..8 (scalar coordinates, no
// runtime-indexed arrays): its lex index, parity, boundary sign, direction
struct PathHop {
  int src, src_parity, mu;
  float sign;
  bool fwd;
};

__device__ __forceinline__ PathHop path_hop(const Geom& g, int x0, int x1, int x2, int x3, int p) {
  PathHop h;
  h.mu = (p - 1) >> 1;
  h.fwd = ((p - 1) & 1) == 0;
  h.sign = 1.f;
  int y0 = x0, y1 = x1, y2 = x2, y3 = x3;
  switch (h.mu) {
    case 0: y0 = h.fwd ? (x0 + 1 == g.L[0] ? 0 : x0 + 1) : (x0 == 0 ? g.L[0] - 1 : x0 - 1); break;
    case 1: y1 = h.fwd ? (x1 + 1 == g.L[1] ? 0 : x1 + 1) : (x1 == 0 ? g.L[1] - 1 : x1 - 1); break;
    case 2: y2 = h.fwd ? (x2 + 1 == g.L[2] ? 0 : x2 + 1) : (x2 == 0 ? g.L[2] - 1 : x2 - 1); break;
    default:
      y3 = h.fwd ? (x3 + 1 == g.L[3] ? 0 : x3 + 1) : (x3 == 0 ? g.L[3] - 1 : x3 - 1);
      if (g.apbc && (h.fwd ? x3 == g.L[3] - 1 : x3 == 0)) h.sign = -1.f;
      break;
  }
  h.src = ((y3 * g.L[2] + y2) * g.L[1] + y1) * g.L[0] + y0;
  h.src_parity = (y0 + y1 + y2 + y3) & 1;
  return h;
}

// the three rows of U_mu at the site with lex index `lex` and parity `par`
__device__ __forceinline__ void net_link_at(const NetGeom& ng, int lex, int par, int mu, cx<float> r[9]) {
  const float4* base = ng.links + (size_t)par * 4 * F32::LN * ng.lstride;
  load_link<F32>(base, ng.lstride, mu, lex >> 1, r);
  third_row(r, r + 6);
}

// effective transport matrix of a hop: w = sign * U (forward) or sign * U^dag
// (backward), so that the transported colour vector is w v in both cases
__device__ __forceinline__ void effective_link(const cx<float> u[9], bool fwd, float sign, cx<float> w[9]) {
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const cx<float> e = fwd ? u[3 * a + b] : cconj(u[3 * b + a]);
      w[3 * a + b] = sign * e;
    }
}

// forward gather: Z rows 3x + a, the column group of path p and channel c.
// One thread per (site, path, channel), channel fastest, so a warp writes
// contiguous 16-byte groups of each row.  blockIdx.y = sample of a batch
// (consecutive 3V-row blocks).
__global__ void __launch_bounds__(NET_NT) pt_gather_kernel(NetGeom ng, const float* __restrict__ X, int C,
                                                          __nv_bfloat16* __restrict__ Z) {
  const int tid = blockIdx.x * NET_NT + threadIdx.x;   // V * 9 * C < 2^31 (checked by the host)
  if (tid >= ng.g.V * PT_PATHS * C) return;
  X += (size_t)blockIdx.y * 3 * ng.g.V * 8 * C;
  Z += (size_t)blockIdx.y * 3 * ng.g.V * 72 * C;
  const int xp = tid / C;
  const int ch = tid - xp * C;
  const int x = xp / PT_PATHS;
  const int p = xp - x * PT_PATHS;
  const Geom& g = ng.g;
  int r = x;
  const int x0 = r % g.L[0];
  r /= g.L[0];
  const int x1 = r % g.L[1];
  r /= g.L[1];
  const int x2 = r % g.L[2];
  const int x3 = r / g.L[2];
  cx<float> v[4][3], out[4][3];
  if (p == 0) {
    load_channel(X, C, x, ch, out);
  } else {
    const PathHop h = path_hop(g, x0, x1, x2, x3, p);
    load_channel(X, C, h.src, ch, v);
    cx<float> u[9], w[9];
    if (h.fwd) net_link_at(ng, x, (x0 + x1 + x2 + x3) & 1, h.mu, u);   // U_mu(x)
    else net_link_at(ng, h.src, h.src_parity, h.mu, u);                // U_mu(x - mu), applied as U^dag
    effective_link(u, h.fwd, h.sign, w);
#pragma unroll
    for (int s2 = 0; s2 < 4; ++s2)
#pragma unroll
      for (int a = 0; a < 3; ++a) out[s2][a] = w[3 * a] * v[s2][0] + w[3 * a + 1] * v[s2][1] + w[3 * a + 2] * v[s2][2];
  }
  const int j8 = (p * C + ch) * 8;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    __nv_bfloat162 r01 = __floats2bfloat162_rn(out[0][a].re, out[1][a].re);
    __nv_bfloat162 r23 = __floats2bfloat162_rn(out[2][a].re, out[3][a].re);
    __nv_bfloat162 i01 = __floats2bfloat162_rn(out[0][a].im, out[1][a].im);
    __nv_bfloat162 i23 = __floats2bfloat162_rn(out[2][a].im, out[3][a].im);
    uint4 q;
    q.x = *reinterpret_cast<uint32_t*>(&r01);
    q.y = *reinterpret_cast<uint32_t*>(&r23);
    q.z = *reinterpret_cast<uint32_t*>(&i01);
    q.w = *reinterpret_cast<uint32_t*>(&i23);
    *reinterpret_cast<uint4*>(Z + (size_t)(3 * x + a) * (72 * C) + j8) = q;
  }
}

// backward gather (adjoint transports): dX(y)_c = sum_p (T_p^dag dZ_{p,c})(y).
// T_p^dag is the transport of the opposite hop of the same direction
// (T_{2mu+1}^dag = T_{2mu+2} and back, same boundary sign), so the neighbour
// and link come from path_hop of the swapped path.
__global__ void __launch_bounds__(NET_NT) pt_gather_adjoint_kernel(NetGeom ng, const float* __restrict__ dZ, int C,
                                                                  float* __restrict__ dX) {
  const int tid = blockIdx.x * NET_NT + threadIdx.x;
  if (tid >= ng.g.V * C) return;
  dZ += (size_t)blockIdx.y * 3 * ng.g.V * 72 * C;
  dX += (size_t)blockIdx.y * 3 * ng.g.V * 8 * C;
  const int y = tid / C;
  const int ch = tid - y * C;
  const int K = 36 * C;
  const Geom& g = ng.g;
  int r = y;
  const int x0 = r % g.L[0];
  r /= g.L[0];
  const int x1 = r % g.L[1];
  r /= g.L[1];
  const int x2 = r % g.L[2];
  const int x3 = r / g.L[2];
  cx<float> acc[4][3];
#pragma unroll
  for (int s2 = 0; s2 < 4; ++s2)
#pragma unroll
    for (int a = 0; a < 3; ++a) acc[s2][a] = {0.f, 0.f};
  for (int p = 0; p < PT_PATHS; ++p) {
    const int j8 = (p * C + ch) * 8;
    int src = y;
    cx<float> w[9];
    if (p > 0) {
      const int q = ((p - 1) & 1) ? p - 1 : p + 1;   // the opposite hop
      const PathHop h = path_hop(g, x0, x1, x2, x3, q);
      src = h.src;
      cx<float> u[9];
      if (h.fwd) net_link_at(ng, y, (x0 + x1 + x2 + x3) & 1, h.mu, u);
      else net_link_at(ng, src, h.src_parity, h.mu, u);
      effective_link(u, h.fwd, h.sign, w);
    }
    cx<float> v[4][3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const float* row = dZ + (size_t)(3 * src + b) * (2 * K) + j8;
      const float4 re = *reinterpret_cast<const float4*>(row);
      const float4 im = *reinterpret_cast<const float4*>(row + 4);
      v[0][b] = {re.x, im.x};
      v[1][b] = {re.y, im.y};
      v[2][b] = {re.z, im.z};
      v[3][b] = {re.w, im.w};
    }
    if (p == 0) {
#pragma unroll
      for (int s2 = 0; s2 < 4; ++s2)
#pragma unroll
        for (int a = 0; a < 3; ++a) acc[s2][a] = acc[s2][a] + v[s2][a];
    } else {
#pragma unroll
      for (int s2 = 0; s2 < 4; ++s2)
#pragma unroll
        for (int a = 0; a < 3; ++a)
          acc[s2][a] = acc[s2][a] + w[3 * a] * v[s2][0] + w[3 * a + 1] * v[s2][1] + w[3 * a + 2] * v[s2][2];
    }
  }
  const int w = 8 * C;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float* row = dX + (size_t)(3 * y + a) * w;
    *reinterpret_cast<float4*>(row + ch * 4) = make_float4(acc[0][a].re, acc[1][a].re, acc[2][a].re, acc[3][a].re);
    *reinterpret_cast<float4*>(row + 4 * C + ch * 4) =
        make_float4(acc[0][a].im, acc[1][a].im, acc[2][a].im, acc[3][a].im);
  }
}

// even-site FP32 parity field (one channel) -> activation with C = 1 (odd
// sites 0); blockIdx.y = sample (parity fields 6 * sstride float4 apart)
__global__ void __launch_bounds__(NET_NT) pt_pack_even_kernel(Geom g, const float4* __restrict__ in, int sstride,
                                                             float* __restrict__ X) {
  const int lex = blockIdx.x * NET_NT + threadIdx.x;
  if (lex >= g.V) return;
  in += (size_t)blockIdx.y * F32::SN * sstride;
  X += (size_t)blockIdx.y * 3 * g.V * 8;
  int c[4];
  lex_coords(g, lex, c);
  cx<float> v[12];
  if (((c[0] + c[1] + c[2] + c[3]) & 1) == 0) {
    load_spinor<F32>(in, sstride, lex >> 1, v);
  } else {
#pragma unroll
    for (int k = 0; k < 12; ++k) v[k] = {0.f, 0.f};
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float* row = X + (size_t)(3 * lex + a) * 8;
    *reinterpret_cast<float4*>(row) = make_float4(v[a].re, v[3 + a].re, v[6 + a].re, v[9 + a].re);
    *reinterpret_cast<float4*>(row + 4) = make_float4(v[a].im, v[3 + a].im, v[6 + a].im, v[9 + a].im);
  }
}

// activation with C = 1 -> even-site FP32 parity field
__global__ void __launch_bounds__(NET_NT) pt_unpack_even_kernel(Geom g, const float* __restrict__ X,
                                                               float4* __restrict__ out, int sstride) {
  const int ih = blockIdx.x * NET_NT + threadIdx.x;
  if (ih >= g.Vh) return;
  X += (size_t)blockIdx.y * 3 * g.V * 8;
  out += (size_t)blockIdx.y * F32::SN * sstride;
  int c[4];
  site_coords(g, 0, ih, c);
  const int lex = lex_of(g, c);
  cx<float> v[12];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float* row = X + (size_t)(3 * lex + a) * 8;
    const float4 re = *reinterpret_cast<const float4*>(row);
    const float4 im = *reinterpret_cast<const float4*>(row + 4);
    v[a] = {re.x, im.x};
    v[3 + a] = {re.y, im.y};
    v[6 + a] = {re.z, im.z};
    v[9 + a] = {re.w, im.w};
  }
  store_spinor<F32>(out, sstride, ih, v);
}

// relative loss per sample on even sites (activations with one channel):
// L = sum_even |y - t|^2 / den, dY = 2 (y - t) / den on even rows, 0 on odd
// rows; the batch total is added to *loss (one atomic per block: reported,
// not used for control).  blockIdx.y = sample.
__global__ void __launch_bounds__(NET_NT) pt_loss_kernel(Geom g, const float* __restrict__ Y,
                                                        const float* __restrict__ T, const double* __restrict__ den,
                                                        float* __restrict__ dY, double* __restrict__ loss) {
  const int lex = blockIdx.x * NET_NT + threadIdx.x;
  const size_t off = (size_t)blockIdx.y * 3 * g.V * 8;
  double part = 0.0;
  if (lex < g.V) {
    int c[4];
    lex_coords(g, lex, c);
    const bool even = ((c[0] + c[1] + c[2] + c[3]) & 1) == 0;
    const float inv = (float)(1.0 / den[blockIdx.y]);
    float s2 = 0.f;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const size_t o = off + (size_t)(3 * lex + r) * 8;
      float d[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        d[e] = even ? Y[o + e] - T[o + e] : 0.f;
        s2 += d[e] * d[e];
      }
      *reinterpret_cast<float4*>(dY + o) = make_float4(2 * inv * d[0], 2 * inv * d[1], 2 * inv * d[2], 2 * inv * d[3]);
      *reinterpret_cast<float4*>(dY + o + 4) =
          make_float4(2 * inv * d[4], 2 * inv * d[5], 2 * inv * d[6], 2 * inv * d[7]);
    }
    part = (double)s2 / den[blockIdx.y];
  }
  __shared__ double sh[NET_NT / 32];
  const double s = block_sum<NET_NT>(part, sh);
  if (threadIdx.x == 0 && loss != nullptr) atomicAdd(loss, s);
}

// sum over even sites of |t|^2 per sample (activation with one channel),
// one atomic per block into den[sample] (den zeroed by the caller)
__global__ void __launch_bounds__(NET_NT) pt_even_norm_kernel(Geom g, const float* __restrict__ T,
                                                             double* __restrict__ den) {
  const int lex = blockIdx.x * NET_NT + threadIdx.x;
  double part = 0.0;
  if (lex < g.V) {
    int c[4];
    lex_coords(g, lex, c);
    if (((c[0] + c[1] + c[2] + c[3]) & 1) == 0) {
      const float* t = T + (size_t)blockIdx.y * 3 * g.V * 8 + (size_t)3 * lex * 8;
      for (int e = 0; e < 24; ++e) part += (double)t[e] * t[e];
    }
  }
  __shared__ double sh[NET_NT / 32];
  const double s = block_sum<NET_NT>(part, sh);
  if (threadIdx.x == 0) atomicAdd(den + blockIdx.y, s);
}

// canonical complex fields [nb][C][V][4][3] (FP64) <-> activations
// [nb][3V][8C] (FP32); one thread per (site, channel), blockIdx.y = sample
__global__ void __launch_bounds__(NET_NT) pt_canon_to_act_kernel(int V, int C, const double2* __restrict__ in,
                                                                float* __restrict__ X) {
  const int tid = blockIdx.x * NET_NT + threadIdx.x;
  if (tid >= V * C) return;
  const int ch = tid / V, lex = tid % V;
  const double2* src = in + ((size_t)blockIdx.y * C + ch) * V * 12 + (size_t)lex * 12;
  float* dst = X + (size_t)blockIdx.y * 3 * V * 8 * C;
  for (int s = 0; s < 4; ++s)
    for (int a = 0; a < 3; ++a) {
      const double2 v = src[3 * s + a];
      float* row = dst + (size_t)(3 * lex + a) * 8 * C;
      row[ch * 4 + s] = (float)v.x;
      row[4 * C + ch * 4 + s] = (float)v.y;
    }
}

__global__ void __launch_bounds__(NET_NT) pt_act_to_canon_kernel(int V, int C, const float* __restrict__ X,
                                                                double2* __restrict__ out) {
  const int tid = blockIdx.x * NET_NT + threadIdx.x;
  if (tid >= V * C) return;
  const int ch = tid / V, lex = tid % V;
  double2* dst = out + ((size_t)blockIdx.y * C + ch) * V * 12 + (size_t)lex * 12;
  const float* src = X + (size_t)blockIdx.y * 3 * V * 8 * C;
  for (int s = 0; s < 4; ++s)
    for (int a = 0; a < 3; ++a) {
      const float* row = src + (size_t)(3 * lex + a) * 8 * C;
      dst[3 * s + a] = make_double2(row[ch * 4 + s], row[4 * C + ch * 4 + s]);
    }
}

// complex FP32 weights [N4][K36] (N4 = 4 C_out, K36 = 36 C_in, column
// kk = 4 j + s) -> BF16 block matrix B [2 N4][72 C_in] in the interleaved
// column layout of Z and its transpose Bt:
//   B[n][8j+s] = Wr, B[n][8j+4+s] = -Wi, B[N4+n][8j+s] = Wi, B[N4+n][8j+4+s] = Wr
__global__ void pt_pack_weights_kernel(const float* __restrict__ wr, const float* __restrict__ wi, int N4, int K36,
                                       __nv_bfloat16* __restrict__ B, __nv_bfloat16* __restrict__ Bt) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= N4 * K36) return;
  const int n = idx / K36, kk = idx % K36;
  const int kr = 2 * kk - (kk & 3), ki = kr + 4;   // 8 (kk / 4) + (kk % 4) and its imaginary slot
  const float r = wr[idx], i = wi[idx];
  const int K2 = 2 * K36, N2 = 2 * N4;
  const __nv_bfloat16 br = __float2bfloat16(r), bi = __float2bfloat16(i), bmi = __float2bfloat16(-i);
  B[(size_t)n * K2 + kr] = br;
  B[(size_t)n * K2 + ki] = bmi;
  B[(size_t)(N4 + n) * K2 + kr] = bi;
  B[(size_t)(N4 + n) * K2 + ki] = br;
  Bt[(size_t)kr * N2 + n] = br;
  Bt[(size_t)ki * N2 + n] = bmi;
  Bt[(size_t)kr * N2 + N4 + n] = bi;
  Bt[(size_t)ki * N2 + N4 + n] = br;
}

// split-K partials of dB^T [splits][72 C_in][2 N4] (dB = dL/dB of the block
// matrix B, interleaved columns) -> complex weight gradient (+=),
// G = dL/dWr + i dL/dWi:
//   dL/dWr = dB[n][8j+s] + dB[N4+n][8j+4+s],  dL/dWi = dB[N4+n][8j+s] - dB[n][8j+4+s]
__global__ void pt_weight_grad_kernel(const float* __restrict__ part, int splits, int N4, int K36,
                                      float* __restrict__ gr, float* __restrict__ gi) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= N4 * K36) return;
  const int n = idx / K36, kk = idx % K36;
  const int kr = 2 * kk - (kk & 3), ki = kr + 4;
  const int N2 = 2 * N4;
  const size_t zs = (size_t)2 * K36 * N2;
  float a = 0.f, b = 0.f, c = 0.f, d = 0.f;
  for (int z = 0; z < splits; ++z) {
    const float* P = part + z * zs;
    a += P[(size_t)kr * N2 + n];
    b += P[(size_t)ki * N2 + N4 + n];
    c += P[(size_t)kr * N2 + N4 + n];
    d += P[(size_t)ki * N2 + n];
  }
  gr[idx] += a + b;
  gi[idx] += c - d;
}

// FP32 -> BF16
__global__ void pt_to_bf16_kernel(const float* __restrict__ in, __nv_bfloat16* __restrict__ out, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = __float2bfloat16(in[i]);
}

// transpose [R][Cc] (FP32 or BF16) -> BF16 [Cc][R] through 32 x 32 shared-memory tiles
template <class T>
__global__ void pt_transpose_kernel(const T* __restrict__ in, int R, int Cc, __nv_bfloat16* __restrict__ out) {
  __shared__ __nv_bfloat16 tile[32][33];
  const int by = blockIdx.x * 32, bx = blockIdx.y * 32;   // rows on grid.x (the long dimension)
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int r = by + j, cc = bx + threadIdx.x;
    if (r < R && cc < Cc) tile[j][threadIdx.x] = __float2bfloat16((float)in[(size_t)r * Cc + cc]);
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int cc = bx + j, r = by + threadIdx.x;
    if (r < R && cc < Cc) out[(size_t)cc * R + r] = tile[threadIdx.x][j];
  }
}

// Adam step on one weight array (Kingma & Ba 2015), gradients cleared after use
__global__ void pt_adam_kernel(float* __restrict__ w, float* __restrict__ g, float* __restrict__ m,
                               float* __restrict__ v, int n, float lr, float b1, float b2, float eps, float c1,
                               float c2, float scale) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i] * scale;
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  g[i] = 0.f;
}

}  // namespace tsm
