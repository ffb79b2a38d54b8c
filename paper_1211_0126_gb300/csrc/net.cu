// net.cu -- the learned LP preconditioner: tensor-core GEMM launches, the
// network object (forward, backward, Adam), training-pair generation from
// the method's own FP32 solves, and the C ABI of the network.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include <cudaTypedefs.h>

#include "contract.h"
#include "net.h"
#include "ptnet.cuh"
#include "solver.h"
#include "umma.cuh"

namespace tsm {

namespace {

template <int BN>
int umma_launch(cudaStream_t stream, dim3 grid, const __nv_bfloat16* A, const __nv_bfloat16* B, float* C, int M,
                int N, int K, int ldc, int beta, int* error, int lda, int ldb, int kchunk, long long czs) {
  const int smem = umma_smem_bytes<BN>();
  if (cudaFuncSetAttribute(umma_gemm_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
    return TSM_ERR_CUDA;
  umma_gemm_kernel<BN><<<grid, UMMA_THREADS, smem, stream>>>(A, B, C, M, N, K, ldc, beta, error, lda, ldb, kchunk,
                                                             czs);
  return cudaGetLastError() == cudaSuccess ? TSM_OK : TSM_ERR_CUDA;
}

// cuTensorMapEncodeTiled from the driver (no link-time dependency on libcuda)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// tensor map of a row-major BF16 matrix [rows][cols] with leading dimension
// ld, read in boxes of 64 columns x box_rows rows with 128-byte swizzle, zero
// fill outside
bool make_tensor_map(CUtensorMap* m, const void* base, int rows, int cols, int ld, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = tensor_map_encoder();
  if (fn == nullptr || (reinterpret_cast<uintptr_t>(base) & 15) != 0) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box[2] = {(cuuint32_t)UMMA_TMA_BOX_K, (cuuint32_t)box_rows};
  const cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool g_umma_tma = true;   // TMA-fed kernel when the operands allow it
std::atomic<int> g_umma_withhold{0};   // fault injection (tsm_umma_inject_timeout)

template <int BN>
int umma_launch_any(cudaStream_t stream, dim3 grid, const __nv_bfloat16* A, const __nv_bfloat16* B, float* C, int M,
                    int N, int K, int ldc, int beta, int* error, int lda, int ldb, int kchunk, long long czs) {
  CUtensorMap ta, tb;
  if (g_umma_tma && make_tensor_map(&ta, A, M, K, lda, UMMA_BM) && make_tensor_map(&tb, B, N, K, ldb, BN)) {
    const int smem = umma_tma_smem_bytes<BN>();
    if (cudaFuncSetAttribute(umma_tma_gemm_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
        cudaSuccess)
      return TSM_ERR_CUDA;
    umma_tma_gemm_kernel<BN><<<grid, UMMA_THREADS, smem, stream>>>(ta, tb, C, M, N, K, ldc, beta, error, kchunk, czs,
                                                                   g_umma_withhold.load());
    return cudaGetLastError() == cudaSuccess ? TSM_OK : TSM_ERR_CUDA;
  }
  return umma_launch<BN>(stream, grid, A, B, C, M, N, K, ldc, beta, error, lda, ldb, kchunk, czs);
}

}  // namespace

// C (FP32) = A (BF16, rows of length lda) * B (BF16, rows of length ldb)^T over
// K columns (+ C if beta).  splits > 1: split-K, partial z written to
// C + z * M * ldc (the caller reduces); *used_splits receives the number of
// partials written (never more than requested).  N is covered by
// ceil(N / 256) tiles of equal width (a multiple of 16).
int launch_umma_gemm_ex(cudaStream_t stream, const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb,
                        float* C, int ldc, int M, int N, int K, int beta, int splits, int* error, int* used_splits) {
  if (used_splits) *used_splits = 0;
  if (M <= 0 || N <= 0) return TSM_OK;
  if (K <= 0 || (K % 8) != 0 || (lda % 8) != 0 || (ldb % 8) != 0 || lda < K || ldb < K) {
    set_error("umma gemm needs K > 0 and K, lda >= K, ldb >= K multiples of 8 (K %d, lda %d, ldb %d)", K, lda, ldb);
    return TSM_ERR_ARG;
  }
  if (splits < 1) splits = 1;
  int kchunk = (K + splits - 1) / splits;
  kchunk = (kchunk + UMMA_BK - 1) / UMMA_BK * UMMA_BK;   // whole stages per split, 16-byte aligned starts
  splits = (K + kchunk - 1) / kchunk;                    // never more than requested
  if (used_splits) *used_splits = splits;
  const long long czs = (long long)M * ldc;
  const int gm = (M + UMMA_BM - 1) / UMMA_BM;
  const int gn = (N + 255) / 256;
  const int w = (N + gn - 1) / gn;
  const dim3 grid(gm, gn, splits);
#define TSM_UMMA_CASE(BN) \
  if (w <= BN) return umma_launch_any<BN>(stream, grid, A, B, C, M, N, K, ldc, beta, error, lda, ldb, kchunk, czs);
  TSM_UMMA_CASE(16)
  TSM_UMMA_CASE(32)
  TSM_UMMA_CASE(48)
  TSM_UMMA_CASE(64)
  TSM_UMMA_CASE(96)
  TSM_UMMA_CASE(128)
  TSM_UMMA_CASE(160)
  TSM_UMMA_CASE(192)
  TSM_UMMA_CASE(224)
  TSM_UMMA_CASE(256)
#undef TSM_UMMA_CASE
  return TSM_ERR_ARG;
}

int launch_umma_gemm(cudaStream_t stream, const __nv_bfloat16* A, const __nv_bfloat16* B, float* C, int M, int N,
                     int K, int ldc, int beta, int* error) {
  return launch_umma_gemm_ex(stream, A, K, B, K, C, ldc, M, N, K, beta, 1, error, nullptr);
}

namespace {

int grid1(long long n, int nt) { return (int)((n + nt - 1) / nt); }

template <class T>
int dalloc(T** p, size_t count) {
  TSM_CUDA(cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(count, 1) * sizeof(T)));
  return TSM_OK;
}

template <class T>
void dfree(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

// splitmix64 (Steele, Lea & Flood 2014) and Box-Muller normals for the
// weight initialisation
struct InitRng {
  uint64_t s;
  uint64_t next() {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  double uniform() { return ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
  double normal() {
    const double u = uniform(), v = uniform();
    return std::sqrt(-2.0 * std::log(u)) * std::cos(6.283185307179586 * v);
  }
};

NetGeom net_geom(const Ctx& c) {
  return NetGeom{c.g, static_cast<const float4*>(c.links[TSM_F32]), c.lstride};
}

int check_net_launch(Ctx& c, const char* what) {
  c.launches++;
  return check_launch(c, what);
}

}  // namespace

int Net::cmax() const {
  int m = 1;
  for (const NetLayer& l : layers) m = std::max(m, std::max(l.cin, l.cout));
  return m;
}

int Net::reserve(int V, int nb) {
  if (V == ws_V && nb <= ws_nb) return TSM_OK;
  if ((long long)V * PT_PATHS * cmax() >= (1ll << 31) || (long long)nb * 3 * V * 8 * cmax() >= (1ll << 40)) {
    set_error("lattice too large for the network kernels (V * 9 * C must stay below 2^31)");
    return TSM_ERR_TOO_LARGE;
  }
  const int L = (int)layers.size();
  for (float*& a : acts) dfree(a);
  dfree(Z);
  dfree(Zt);
  dfree(dZ);
  dfree(dA[0]);
  dfree(dA[1]);
  dfree(dYb);
  dfree(dYt);
  const size_t M = (size_t)nb * 3 * V;
  const int cm = cmax();
  acts.assign(L + 1, nullptr);
  for (int l = 1; l <= L; ++l) TSM_TRY(dalloc(&acts[l], M * 8 * layers[l - 1].cout));
  TSM_TRY(dalloc(&Z, M * 72 * cm));
  TSM_TRY(dalloc(&Zt, M * 72 * cm));
  TSM_TRY(dalloc(&dZ, M * 72 * cm));
  TSM_TRY(dalloc(&dA[0], M * 8 * cm));
  TSM_TRY(dalloc(&dA[1], M * 8 * cm));
  TSM_TRY(dalloc(&dYb, M * 8 * cm));
  TSM_TRY(dalloc(&dYt, M * 8 * cm));
  ws_V = V;
  ws_nb = nb;
  return TSM_OK;
}

int Net::pack(cudaStream_t s) {
  if (packed) return TSM_OK;
  for (NetLayer& l : layers) {
    const int n = l.n4() * l.k36();
    pt_pack_weights_kernel<<<grid1(n, 256), 256, 0, s>>>(l.wr, l.wi, l.n4(), l.k36(), l.B, l.Bt);
    TSM_CUDA(cudaGetLastError());
  }
  packed = true;
  return TSM_OK;
}

int Net::forward(Ctx& c, const float* X0, int nb, float** out) {
  TSM_TRY(reserve(c.g.V, nb));
  TSM_TRY(pack(c.stream));
  const NetGeom ng = net_geom(c);
  const int V = c.g.V, M = nb * 3 * V;
  const float* X = X0;
  for (size_t li = 0; li < layers.size(); ++li) {
    const NetLayer& l = layers[li];
    const int K2 = 72 * l.cin, N2 = 8 * l.cout;
    pt_gather_kernel<<<dim3(grid1((long long)V * PT_PATHS * l.cin, NET_NT), nb), NET_NT, 0, c.stream>>>(ng, X, l.cin,
                                                                                                        Z);
    TSM_TRY(check_net_launch(c, "pt_gather_kernel"));
    TSM_TRY(launch_umma_gemm_ex(c.stream, Z, K2, l.B, K2, acts[li + 1], N2, M, N2, K2, 0, 1, d_err, nullptr));
    TSM_TRY(check_net_launch(c, "umma_gemm_kernel"));
    X = acts[li + 1];
  }
  *out = acts[layers.size()];
  return TSM_OK;
}

int Net::backward(Ctx& c, const float* X0, int nb, const float* dY, float* dX0) {
  const NetGeom ng = net_geom(c);
  const int V = c.g.V, M = nb * 3 * V;
  const float* g = dY;
  int cur = 0;
  for (int li = (int)layers.size() - 1; li >= 0; --li) {
    NetLayer& l = layers[li];
    const int K2 = 72 * l.cin, N2 = 8 * l.cout;
    const float* X = li == 0 ? X0 : acts[li];
    // output gradient in BF16, row-major and transposed
    pt_to_bf16_kernel<<<grid1((long long)M * N2, 256), 256, 0, c.stream>>>(g, dYb, (long long)M * N2);
    TSM_TRY(check_net_launch(c, "pt_to_bf16_kernel"));
    pt_transpose_kernel<float><<<dim3(grid1(M, 32), grid1(N2, 32)), dim3(32, 8), 0, c.stream>>>(g, M, N2, dYt);
    TSM_TRY(check_net_launch(c, "pt_transpose_kernel"));
    // gathered input and its transpose
    pt_gather_kernel<<<dim3(grid1((long long)V * PT_PATHS * l.cin, NET_NT), nb), NET_NT, 0, c.stream>>>(ng, X, l.cin,
                                                                                                        Z);
    TSM_TRY(check_net_launch(c, "pt_gather_kernel"));
    pt_transpose_kernel<__nv_bfloat16><<<dim3(grid1(M, 32), grid1(K2, 32)), dim3(32, 8), 0, c.stream>>>(Z, M, K2,
                                                                                                          Zt);
    TSM_TRY(check_net_launch(c, "pt_transpose_kernel"));
    // dB^T = Z^T dY, split over the rows (sites x colours)
    const int tiles = grid1(K2, UMMA_BM) * grid1(N2, 256);
    int splits = std::max(1, std::min(2 * 152 / tiles, grid1(M, 4 * UMMA_BK)));
    const size_t need = (size_t)splits * K2 * N2;
    if (need > part_cap) {
      dfree(part);
      TSM_TRY(dalloc(&part, need));
      part_cap = need;
    }
    TSM_TRY(launch_umma_gemm_ex(c.stream, Zt, M, dYt, M, part, N2, K2, N2, M, 0, splits, d_err, &splits));
    TSM_TRY(check_net_launch(c, "umma_gemm_kernel"));
    pt_weight_grad_kernel<<<grid1(l.n4() * l.k36(), 256), 256, 0, c.stream>>>(part, splits, l.n4(), l.k36(), l.gr,
                                                                              l.gi);
    TSM_TRY(check_net_launch(c, "pt_weight_grad_kernel"));
    if (li == 0 && dX0 == nullptr) break;
    // dZ = dY B, then the adjoint transports give the input gradient
    TSM_TRY(launch_umma_gemm_ex(c.stream, dYb, N2, l.Bt, N2, dZ, K2, M, K2, N2, 0, 1, d_err, nullptr));
    TSM_TRY(check_net_launch(c, "umma_gemm_kernel"));
    float* dst = li > 0 ? dA[cur] : dX0;
    pt_gather_adjoint_kernel<<<dim3(grid1((long long)V * l.cin, NET_NT), nb), NET_NT, 0, c.stream>>>(ng, dZ, l.cin,
                                                                                                    dst);
    TSM_TRY(check_net_launch(c, "pt_gather_adjoint_kernel"));
    g = dst;
    cur ^= 1;
  }
  return TSM_OK;
}

void Net::free_all() {
  for (NetLayer& l : layers) {
    dfree(l.wr);
    dfree(l.wi);
    dfree(l.gr);
    dfree(l.gi);
    dfree(l.mr);
    dfree(l.vr);
    dfree(l.mi);
    dfree(l.vi);
    dfree(l.B);
    dfree(l.Bt);
  }
  for (PairGroup& g : groups) {
    dfree(g.R);
    dfree(g.T);
    dfree(g.den);
  }
  for (float*& a : acts) dfree(a);
  dfree(Z);
  dfree(Zt);
  dfree(dZ);
  dfree(dA[0]);
  dfree(dA[1]);
  dfree(dYb);
  dfree(dYt);
  dfree(part);
  dfree(d_err);
  dfree(d_loss);
  ws_V = ws_nb = 0;
}

int net_apply_even(Ctx& c, Net& n, const PField& in, const PField& out, int nrhs) {
  TSM_TRY(n.reserve(c.g.V, nrhs));
  float* X0 = n.dA[0];   // input activation (free outside the backward pass)
  pt_pack_even_kernel<<<dim3(grid1(c.g.V, NET_NT), nrhs), NET_NT, 0, c.stream>>>(c.g, in.as<F32>(), c.sstride, X0);
  TSM_TRY(check_net_launch(c, "pt_pack_even_kernel"));
  float* Y = nullptr;
  TSM_TRY(n.forward(c, X0, nrhs, &Y));
  pt_unpack_even_kernel<<<dim3(grid1(c.g.Vh, NET_NT), nrhs), NET_NT, 0, c.stream>>>(c.g, Y, out.as<F32>(),
                                                                                    c.sstride);
  return check_net_launch(c, "pt_unpack_even_kernel");
}

}  // namespace tsm

using namespace tsm;

namespace {

int nbad(int code, const char* msg) {
  set_error("%s", msg);
  return code;
}

int check_timeout(Net& n, cudaStream_t s) {
  int herr = 0;
  TSM_CUDA(cudaMemcpyAsync(&herr, n.d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  TSM_CUDA(cudaStreamSynchronize(s));
  if (herr) {
    set_error("a tensor-core wait of the network timed out");
    return TSM_ERR_TIMEOUT;
  }
  return TSM_OK;
}

int check_ctx(tsm_ctx* h, const Net& n) {
  if (h == nullptr) return nbad(TSM_ERR_ARG, "null context");
  if (!h->c.has_gauge) return nbad(TSM_ERR_NO_GAUGE, "no gauge field loaded");
  if (h->c.device != n.device) return nbad(TSM_ERR_ARG, "network and context live on different devices");
  TSM_CUDA(cudaSetDevice(n.device));
  return TSM_OK;
}

int adam_step(Net& n, cudaStream_t s, double lr, double scale) {
  n.adam_t++;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = 1.f - std::pow(b1, (float)n.adam_t), c2 = 1.f - std::pow(b2, (float)n.adam_t);
  for (NetLayer& l : n.layers) {
    const int cnt = l.n4() * l.k36();
    pt_adam_kernel<<<grid1(cnt, 256), 256, 0, s>>>(l.wr, l.gr, l.mr, l.vr, cnt, (float)lr, b1, b2, eps, c1, c2,
                                                   (float)scale);
    pt_adam_kernel<<<grid1(cnt, 256), 256, 0, s>>>(l.wi, l.gi, l.mi, l.vi, cnt, (float)lr, b1, b2, eps, c1, c2,
                                                   (float)scale);
    TSM_CUDA(cudaGetLastError());
  }
  n.packed = false;
  return TSM_OK;
}

int zero_grads(Net& n, cudaStream_t s) {
  for (NetLayer& l : n.layers) {
    const size_t b = (size_t)l.n4() * l.k36() * sizeof(float);
    TSM_CUDA(cudaMemsetAsync(l.gr, 0, b, s));
    TSM_CUDA(cudaMemsetAsync(l.gi, 0, b, s));
  }
  return TSM_OK;
}

}  // namespace

extern "C" int tsm_umma_gemm_ex(const void* A, int lda, const void* B, int ldb, float* C, int ldc, int M, int N,
                                int K, int beta, int splits, int* used_splits, void* cuda_stream) {
  if (A == nullptr || B == nullptr || C == nullptr) return nbad(TSM_ERR_ARG, "tsm_umma_gemm: null argument");
  if (ldc < N) return nbad(TSM_ERR_ARG, "tsm_umma_gemm: ldc < N");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  int* err = nullptr;
  TSM_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&err), sizeof(int), s));
  TSM_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
  int used = 0;
  int rc = launch_umma_gemm_ex(s, static_cast<const __nv_bfloat16*>(A), lda, static_cast<const __nv_bfloat16*>(B), ldb,
                               C, ldc, M, N, K, beta, splits, err, &used);
  int herr = 0;
  if (rc == TSM_OK) {
    TSM_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    TSM_CUDA(cudaStreamSynchronize(s));
  }
  cudaFreeAsync(err, s);
  if (used_splits) *used_splits = used;
  if (rc != TSM_OK) {
    if (rc == TSM_ERR_CUDA) set_error("tsm_umma_gemm: launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    return rc;
  }
  if (herr) return nbad(TSM_ERR_TIMEOUT, "tsm_umma_gemm: a tensor-core wait timed out");
  return TSM_OK;
}

extern "C" int tsm_umma_inject_timeout(int withhold) {
  g_umma_withhold.store(withhold ? 1 : 0);
  return TSM_OK;
}

extern "C" int tsm_umma_gemm(const void* A, const void* B, float* C, int M, int N, int K, int beta,
                             void* cuda_stream) {
  return tsm_umma_gemm_ex(A, K, B, K, C, N, M, N, K, beta, 1, nullptr, cuda_stream);
}

extern "C" int tsm_net_create(int device, int n_layers, const int* channels, uint64_t seed, double init_scale,
                              tsm_net** out) {
  if (out == nullptr || channels == nullptr) return nbad(TSM_ERR_ARG, "null argument");
  *out = nullptr;
  if (n_layers < 1 || n_layers > 16) return nbad(TSM_ERR_ARG, "n_layers must be in [1, 16]");
  if (channels[0] != 1 || channels[n_layers] != 1)
    return nbad(TSM_ERR_ARG, "the first and last channel counts must be 1 (a spinor field in and out)");
  for (int l = 0; l <= n_layers; ++l)
    if (channels[l] < 1 || channels[l] > 64) return nbad(TSM_ERR_ARG, "channel counts must be in [1, 64]");
  TSM_CUDA(cudaSetDevice(device));
  tsm_net* h = new (std::nothrow) tsm_net;
  if (h == nullptr) return nbad(TSM_ERR_ARG, "out of host memory");
  Net& n = h->n;
  n.device = device;
  InitRng rng{seed};
  int rc = TSM_OK;
  n.layers.resize(n_layers);
  for (int li = 0; li < n_layers && rc == TSM_OK; ++li) {
    NetLayer& l = n.layers[li];
    l.cin = channels[li];
    l.cout = channels[li + 1];
    const size_t cnt = (size_t)l.n4() * l.k36();
    float** arrs[] = {&l.wr, &l.wi, &l.gr, &l.gi, &l.mr, &l.vr, &l.mi, &l.vi};
    for (float** a : arrs)
      if (rc == TSM_OK) rc = dalloc(a, cnt);
    if (rc == TSM_OK) rc = dalloc(&l.B, 4 * cnt);
    if (rc == TSM_OK) rc = dalloc(&l.Bt, 4 * cnt);
    if (rc != TSM_OK) break;
    for (float** a : arrs)
      if (*a != l.wr && *a != l.wi && cudaMemset(*a, 0, cnt * sizeof(float)) != cudaSuccess) rc = TSM_ERR_CUDA;
    // near-identity start: channel c' copies channel c' mod C_in on the
    // identity path (the last layer averages its inputs), plus small noise
    std::vector<float> wr(cnt), wi(cnt);
    const double sigma = init_scale / std::sqrt(36.0 * l.cin);
    for (size_t i = 0; i < cnt; ++i) {
      wr[i] = (float)(sigma * rng.normal());
      wi[i] = (float)(sigma * rng.normal());
    }
    for (int co = 0; co < l.cout; ++co)
      for (int s = 0; s < 4; ++s) {
        if (l.cout == 1) {
          for (int ci = 0; ci < l.cin; ++ci) wr[(size_t)(co * 4 + s) * l.k36() + ci * 4 + s] += 1.f / l.cin;
        } else {
          const int ci = co % l.cin;
          wr[(size_t)(co * 4 + s) * l.k36() + ci * 4 + s] += 1.f;
        }
      }
    if (rc == TSM_OK && cudaMemcpy(l.wr, wr.data(), cnt * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
      rc = TSM_ERR_CUDA;
    if (rc == TSM_OK && cudaMemcpy(l.wi, wi.data(), cnt * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
      rc = TSM_ERR_CUDA;
  }
  if (rc == TSM_OK) rc = dalloc(&n.d_err, 1);
  if (rc == TSM_OK && cudaMemset(n.d_err, 0, sizeof(int)) != cudaSuccess) rc = TSM_ERR_CUDA;
  if (rc != TSM_OK) {
    n.free_all();
    delete h;
    set_error("tsm_net_create: device allocation failed");
    return rc;
  }
  *out = h;
  return TSM_OK;
}

extern "C" int tsm_net_destroy(tsm_net* h) {
  if (h == nullptr) return TSM_OK;
  cudaSetDevice(h->n.device);
  cudaDeviceSynchronize();
  h->n.free_all();
  delete h;
  return TSM_OK;
}

extern "C" int tsm_net_set_weights(tsm_net* h, int layer, const double* W) {
  if (h == nullptr || W == nullptr) return nbad(TSM_ERR_ARG, "null argument");
  Net& n = h->n;
  if (layer < 0 || layer >= (int)n.layers.size()) return nbad(TSM_ERR_ARG, "layer out of range");
  NetLayer& l = n.layers[layer];
  const size_t cnt = (size_t)l.n4() * l.k36();
  std::vector<float> wr(cnt), wi(cnt);
  for (size_t i = 0; i < cnt; ++i) {
    wr[i] = (float)W[2 * i];
    wi[i] = (float)W[2 * i + 1];
  }
  TSM_CUDA(cudaSetDevice(n.device));
  TSM_CUDA(cudaDeviceSynchronize());
  TSM_CUDA(cudaMemcpy(l.wr, wr.data(), cnt * sizeof(float), cudaMemcpyHostToDevice));
  TSM_CUDA(cudaMemcpy(l.wi, wi.data(), cnt * sizeof(float), cudaMemcpyHostToDevice));
  n.packed = false;
  return TSM_OK;
}

extern "C" int tsm_net_get_weights(tsm_net* h, int layer, double* W) {
  if (h == nullptr || W == nullptr) return nbad(TSM_ERR_ARG, "null argument");
  Net& n = h->n;
  if (layer < 0 || layer >= (int)n.layers.size()) return nbad(TSM_ERR_ARG, "layer out of range");
  NetLayer& l = n.layers[layer];
  const size_t cnt = (size_t)l.n4() * l.k36();
  std::vector<float> wr(cnt), wi(cnt);
  TSM_CUDA(cudaSetDevice(n.device));
  TSM_CUDA(cudaDeviceSynchronize());
  TSM_CUDA(cudaMemcpy(wr.data(), l.wr, cnt * sizeof(float), cudaMemcpyDeviceToHost));
  TSM_CUDA(cudaMemcpy(wi.data(), l.wi, cnt * sizeof(float), cudaMemcpyDeviceToHost));
  for (size_t i = 0; i < cnt; ++i) {
    W[2 * i] = wr[i];
    W[2 * i + 1] = wi[i];
  }
  return TSM_OK;
}

// forward of nb multi-channel canonical fields (marshalling kernels + the path)
extern "C" int tsm_net_forward(tsm_net* h, tsm_ctx* ch, int nb, const double* x, double* y, int on_device) {
  if (h == nullptr || x == nullptr || y == nullptr) return nbad(TSM_ERR_ARG, "null argument");
  if (nb < 1) return nbad(TSM_ERR_ARG, "nb < 1");
  Net& n = h->n;
  TSM_TRY(check_ctx(ch, n));
  Ctx& c = ch->c;
  const int V = c.g.V, C0 = n.layers.front().cin, CL = n.layers.back().cout;
  const size_t in_b = (size_t)nb * C0 * V * 24 * sizeof(double), out_b = (size_t)nb * CL * V * 24 * sizeof(double);
  TSM_TRY(n.reserve(V, nb));
  void *din = const_cast<double*>(x), *dout = y;
  if (!on_device) {
    TSM_TRY(c.buffer("net_io_in", in_b, &din));
    TSM_TRY(c.buffer("net_io_out", out_b, &dout));
    TSM_CUDA(cudaMemcpyAsync(din, x, in_b, cudaMemcpyHostToDevice, c.stream));
  }
  float* X0 = n.dA[0];
  pt_canon_to_act_kernel<<<dim3(grid1((long long)V * C0, NET_NT), nb), NET_NT, 0, c.stream>>>(
      V, C0, static_cast<const double2*>(din), X0);
  TSM_TRY(check_net_launch(c, "pt_canon_to_act_kernel"));
  float* Y = nullptr;
  TSM_TRY(n.forward(c, X0, nb, &Y));
  pt_act_to_canon_kernel<<<dim3(grid1((long long)V * CL, NET_NT), nb), NET_NT, 0, c.stream>>>(
      V, CL, Y, static_cast<double2*>(dout));
  TSM_TRY(check_net_launch(c, "pt_act_to_canon_kernel"));
  if (!on_device) TSM_CUDA(cudaMemcpyAsync(y, dout, out_b, cudaMemcpyDeviceToHost, c.stream));
  return check_timeout(n, c.stream);
}

// input and weight gradients for a given output gradient gy (G = dL/dRe + i dL/dIm)
extern "C" int tsm_net_gradient(tsm_net* h, tsm_ctx* ch, int nb, const double* x, const double* gy, double* gx,
                                double* gw) {
  if (h == nullptr || x == nullptr || gy == nullptr) return nbad(TSM_ERR_ARG, "null argument");
  if (nb < 1) return nbad(TSM_ERR_ARG, "nb < 1");
  Net& n = h->n;
  TSM_TRY(check_ctx(ch, n));
  Ctx& c = ch->c;
  const int V = c.g.V, C0 = n.layers.front().cin, CL = n.layers.back().cout;
  const size_t in_b = (size_t)nb * C0 * V * 24 * sizeof(double), out_b = (size_t)nb * CL * V * 24 * sizeof(double);
  TSM_TRY(n.reserve(V, nb));
  void *dx = nullptr, *dgy = nullptr, *dgx = nullptr, *x0 = nullptr, *gx0 = nullptr;
  TSM_TRY(c.buffer("net_io_in", in_b, &dx));
  TSM_TRY(c.buffer("net_io_out", out_b, &dgy));
  TSM_TRY(c.buffer("net_io_gx", in_b, &dgx));
  TSM_TRY(c.buffer("net_x0", (size_t)nb * 3 * V * 8 * C0 * sizeof(float), &x0));
  TSM_TRY(c.buffer("net_gx0", (size_t)nb * 3 * V * 8 * C0 * sizeof(float), &gx0));
  TSM_CUDA(cudaMemcpyAsync(dx, x, in_b, cudaMemcpyHostToDevice, c.stream));
  TSM_CUDA(cudaMemcpyAsync(dgy, gy, out_b, cudaMemcpyHostToDevice, c.stream));
  TSM_TRY(zero_grads(n, c.stream));
  float* X0 = static_cast<float*>(x0);
  pt_canon_to_act_kernel<<<dim3(grid1((long long)V * C0, NET_NT), nb), NET_NT, 0, c.stream>>>(
      V, C0, static_cast<const double2*>(dx), X0);
  TSM_TRY(check_net_launch(c, "pt_canon_to_act_kernel"));
  float* Y = nullptr;
  TSM_TRY(n.forward(c, X0, nb, &Y));
  pt_canon_to_act_kernel<<<dim3(grid1((long long)V * CL, NET_NT), nb), NET_NT, 0, c.stream>>>(
      V, CL, static_cast<const double2*>(dgy), n.dA[1]);
  TSM_TRY(check_net_launch(c, "pt_canon_to_act_kernel"));
  TSM_TRY(n.backward(c, X0, nb, n.dA[1], static_cast<float*>(gx0)));
  if (gx) {
    pt_act_to_canon_kernel<<<dim3(grid1((long long)V * C0, NET_NT), nb), NET_NT, 0, c.stream>>>(
        V, C0, static_cast<const float*>(gx0), static_cast<double2*>(dgx));
    TSM_TRY(check_net_launch(c, "pt_act_to_canon_kernel"));
    TSM_CUDA(cudaMemcpyAsync(gx, dgx, in_b, cudaMemcpyDeviceToHost, c.stream));
  }
  TSM_TRY(check_timeout(n, c.stream));
  if (gw) {
    size_t off = 0;
    for (NetLayer& l : n.layers) {
      const size_t cnt = (size_t)l.n4() * l.k36();
      std::vector<float> gr(cnt), gi(cnt);
      TSM_CUDA(cudaMemcpy(gr.data(), l.gr, cnt * sizeof(float), cudaMemcpyDeviceToHost));
      TSM_CUDA(cudaMemcpy(gi.data(), l.gi, cnt * sizeof(float), cudaMemcpyDeviceToHost));
      for (size_t i = 0; i < cnt; ++i) {
        gw[2 * (off + i)] = gr[i];
        gw[2 * (off + i) + 1] = gi[i];
      }
      off += cnt;
    }
  }
  return zero_grads(n, c.stream);
}

// n training pairs (r, Dhat^-1 r) of the context's gauge field: r = Z4 noise
// on the even sites (source indices 0 .. n-1 of `seed`), Dhat^-1 r from
// batched FP32 CG solves of the full system with b_e = A r, b_o = 0 (whose
// Schur source is exactly r).
extern "C" int tsm_net_add_pairs(tsm_net* h, tsm_ctx* ch, int n_pairs, uint64_t seed, const tm_stop* stop,
                                 int* group) {
  if (h == nullptr || stop == nullptr) return nbad(TSM_ERR_ARG, "null argument");
  if (n_pairs < 1) return nbad(TSM_ERR_ARG, "n_pairs < 1");
  if (stop->prec != TSM_F32 || stop->reliable || stop->precond)
    return nbad(TSM_ERR_ARG, "training pairs come from plain FP32 solves (prec TSM_F32, no reliable updates)");
  Net& n = h->n;
  TSM_TRY(check_ctx(ch, n));
  Ctx& c = ch->c;
  const int V = c.g.V, Vh = c.g.Vh;
  PairGroup G;
  G.ctx = &c;
  G.n = n_pairs;
  TSM_TRY(dalloc(&G.R, (size_t)n_pairs * 3 * V * 8));
  TSM_TRY(dalloc(&G.T, (size_t)n_pairs * 3 * V * 8));
  TSM_TRY(dalloc(&G.den, n_pairs));
  TSM_CUDA(cudaMemsetAsync(G.den, 0, n_pairs * sizeof(double), c.stream));
  const int width = std::min(n_pairs, Ctx::kMaxBatch);
  c.batch_cap = std::max(c.batch_cap, width);
  PField eta, be, bo, se, so;
  TSM_TRY(c.field("np_eta", TSM_F32, &eta, c.batch_cap));
  TSM_TRY(c.field("np_be", TSM_F32, &be, c.batch_cap));
  TSM_TRY(c.field("np_bo", TSM_F32, &bo, c.batch_cap));
  TSM_TRY(c.field("np_se", TSM_F32, &se, c.batch_cap));
  TSM_TRY(c.field("np_so", TSM_F32, &so, c.batch_cap));
  const NoiseSpec ns = make_noise(seed, 4);
  std::vector<SolveResult> res(width);
  tm_stop st = *stop;
  for (int j0 = 0; j0 < n_pairs; j0 += width) {
    const int m = std::min(width, n_pairs - j0);
    TSM_TRY(launch_noise<F32>(c, 0, ns, (uint32_t)j0, eta, m));
    TSM_TRY(launch_twist<F32>(c, twist_A(c.lat.kappa, c.lat.mu), eta, be, nullptr, nullptr, m));
    TSM_TRY((launch_convert<F32, F32>(c, PField{}, bo, nullptr, m)));
    TSM_TRY(solve_batch(c, st, 0, m, EOField{be, bo}, EOField{se, so}, res.data()));
    for (int r = 0; r < m; ++r)
      if (res[r].status != TSM_OK) return nbad(TSM_ERR_NONFINITE, "a training-pair solve met NaN/Inf");
    const size_t off = (size_t)j0 * 3 * V * 8;
    pt_pack_even_kernel<<<dim3(grid1(V, NET_NT), m), NET_NT, 0, c.stream>>>(c.g, eta.as<F32>(), c.sstride, G.R + off);
    TSM_TRY(check_net_launch(c, "pt_pack_even_kernel"));
    pt_pack_even_kernel<<<dim3(grid1(V, NET_NT), m), NET_NT, 0, c.stream>>>(c.g, se.as<F32>(), c.sstride, G.T + off);
    TSM_TRY(check_net_launch(c, "pt_pack_even_kernel"));
    pt_even_norm_kernel<<<dim3(grid1(V, NET_NT), m), NET_NT, 0, c.stream>>>(c.g, G.T + off, G.den + j0);
    TSM_TRY(check_net_launch(c, "pt_even_norm_kernel"));
  }
  (void)Vh;
  TSM_CUDA(cudaStreamSynchronize(c.stream));
  n.groups.push_back(G);
  if (group) *group = (int)n.groups.size() - 1;
  return TSM_OK;
}

namespace tsm {
namespace {

// out = a - b over n float4 words (batches of FP32 parity fields)
__global__ void sub_f4_kernel(long long n, const float4* __restrict__ a, const float4* __restrict__ b,
                              float4* __restrict__ out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 x = a[i], y = b[i];
  out[i] = make_float4(x.x - y.x, x.y - y.y, x.z - y.z, x.w - y.w);
}

// out_e = Dhat in_e for m even-site FP32 fields (odd scratch u):
// u = A^-1 H_oe in, out = A^-1 (A in - kappa^2 H_eo u)
int schur_f32(Ctx& c, PField in, PField u, PField out, int m) {
  const double k = c.lat.kappa, mu = c.lat.mu;
  HopArgs<F32> h = hop_args<F32>(c, 1);
  h.in = in.as<F32>();
  h.out = u.as<F32>();
  h.to = twist_Ainv(k, mu);
  TSM_TRY(launch_hop<F32>(c, h, 0, 0, -1, m));
  h = hop_args<F32>(c, 0);
  h.in = u.as<F32>();
  h.center = in.as<F32>();
  h.tc = twist_A(k, mu);
  h.ac = 1.0;
  h.ah = -k * k;
  h.to = twist_Ainv(k, mu);
  h.out = out.as<F32>();
  return launch_hop<F32>(c, h, 0, HOP_CENTER, -1, m);
}

}  // namespace
}  // namespace tsm

extern "C" int tsm_net_add_solve_pairs(tsm_net* h, tsm_ctx* ch, int n_sources, uint64_t seed, const int* iters,
                                       int n_iters, const tm_stop* stop, int* group) {
  if (h == nullptr || stop == nullptr || iters == nullptr) return nbad(TSM_ERR_ARG, "null argument");
  if (n_sources < 1 || n_iters < 1) return nbad(TSM_ERR_ARG, "n_sources and n_iters must be >= 1");
  if (stop->prec != TSM_F32 || stop->reliable || stop->precond)
    return nbad(TSM_ERR_ARG, "training solves are plain FP32 CG (prec TSM_F32, no reliable updates)");
  for (int q = 0; q < n_iters; ++q)
    if (iters[q] < 0) return nbad(TSM_ERR_ARG, "iteration counts must be >= 0");
  Net& n = h->n;
  TSM_TRY(check_ctx(ch, n));
  Ctx& c = ch->c;
  const int V = c.g.V;
  const int n_pairs = n_sources * n_iters;
  PairGroup G;
  G.ctx = &c;
  G.n = n_pairs;
  TSM_TRY(dalloc(&G.R, (size_t)n_pairs * 3 * V * 8));
  TSM_TRY(dalloc(&G.T, (size_t)n_pairs * 3 * V * 8));
  TSM_TRY(dalloc(&G.den, n_pairs));
  TSM_CUDA(cudaMemsetAsync(G.den, 0, n_pairs * sizeof(double), c.stream));
  const int width = std::min(n_sources, Ctx::kMaxBatch);
  c.batch_cap = std::max(c.batch_cap, width);
  PField bo, be, xe, xo, ke, ko, te, ue, re;
  TSM_TRY(c.field("sp_be", TSM_F32, &be, c.batch_cap));
  TSM_TRY(c.field("sp_bo", TSM_F32, &bo, c.batch_cap));
  TSM_TRY(c.field("sp_xe", TSM_F32, &xe, c.batch_cap));
  TSM_TRY(c.field("sp_xo", TSM_F32, &xo, c.batch_cap));
  TSM_TRY(c.field("sp_ke", TSM_F32, &ke, c.batch_cap));
  TSM_TRY(c.field("sp_ko", TSM_F32, &ko, c.batch_cap));
  TSM_TRY(c.field("sp_te", TSM_F32, &te, c.batch_cap));
  TSM_TRY(c.field("sp_ue", TSM_F32, &ue, c.batch_cap));
  TSM_TRY(c.field("sp_re", TSM_F32, &re, c.batch_cap));
  const NoiseSpec ns = make_noise(seed, 4);
  std::vector<SolveResult> res(width);
  for (int j0 = 0; j0 < n_sources; j0 += width) {
    const int m = std::min(width, n_sources - j0);
    // sources eta_j as tsm_loops draws them; the converged solution x*
    TSM_TRY(launch_noise<F32>(c, 0, ns, (uint32_t)j0, be, m));
    TSM_TRY(launch_noise<F32>(c, 1, ns, (uint32_t)j0, bo, m));
    TSM_TRY(solve_batch(c, *stop, 0, m, EOField{be, bo}, EOField{xe, xo}, res.data()));
    for (int r = 0; r < m; ++r)
      if (res[r].status != TSM_OK) return nbad(TSM_ERR_NONFINITE, "a training solve met NaN/Inf");
    for (int q = 0; q < n_iters; ++q) {
      // the iterate after iters[q] CGNR iterations from zero (the first
      // iterations of the same solve), t = x* - x_k, r = Dhat t
      if (iters[q] == 0) {
        TSM_TRY((launch_convert<F32, F32>(c, PField{}, ke, nullptr, m)));   // x_0 = 0: t = x*, r = bhat
      } else {
        const tm_stop sk{0.0, iters[q], TSM_F32, 0, 0.0, 0, 0};
        TSM_TRY(solve_batch(c, sk, 0, m, EOField{be, bo}, EOField{ke, ko}, res.data()));
      }
      const long long n4 = (long long)m * F32::SN * c.sstride;
      sub_f4_kernel<<<(unsigned)((n4 + 255) / 256), 256, 0, c.stream>>>(n4, xe.as<F32>(), ke.as<F32>(), te.as<F32>());
      TSM_TRY(check_net_launch(c, "sub_f4_kernel"));
      TSM_TRY(schur_f32(c, te, ue, re, m));
      const size_t off = ((size_t)j0 * n_iters + (size_t)q * m) * 3 * V * 8;
      const int p0 = j0 * n_iters + q * m;
      pt_pack_even_kernel<<<dim3(grid1(V, NET_NT), m), NET_NT, 0, c.stream>>>(c.g, re.as<F32>(), c.sstride, G.R + off);
      TSM_TRY(check_net_launch(c, "pt_pack_even_kernel"));
      pt_pack_even_kernel<<<dim3(grid1(V, NET_NT), m), NET_NT, 0, c.stream>>>(c.g, te.as<F32>(), c.sstride, G.T + off);
      TSM_TRY(check_net_launch(c, "pt_pack_even_kernel"));
      pt_even_norm_kernel<<<dim3(grid1(V, NET_NT), m), NET_NT, 0, c.stream>>>(c.g, G.T + off, G.den + p0);
      TSM_TRY(check_net_launch(c, "pt_even_norm_kernel"));
    }
  }
  std::vector<double> den(n_pairs);
  TSM_CUDA(cudaMemcpyAsync(den.data(), G.den, n_pairs * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  TSM_CUDA(cudaStreamSynchronize(c.stream));
  for (int p = 0; p < n_pairs; ++p)
    if (!(den[p] > 0.0)) {
      dfree(G.R);
      dfree(G.T);
      dfree(G.den);
      return nbad(TSM_ERR_ARG, "an iterate equals the converged solution (iteration count too large)");
    }
  n.groups.push_back(G);
  if (group) *group = (int)n.groups.size() - 1;
  return TSM_OK;
}

extern "C" int tsm_net_get_pair(tsm_net* h, int group, int index, double* r, double* t) {
  if (h == nullptr || r == nullptr || t == nullptr) return nbad(TSM_ERR_ARG, "null argument");
  Net& n = h->n;
  if (group < 0 || group >= (int)n.groups.size()) return nbad(TSM_ERR_ARG, "no such pair group");
  PairGroup& G = n.groups[group];
  if (index < 0 || index >= G.n) return nbad(TSM_ERR_ARG, "pair index out of range");
  Ctx& c = *G.ctx;
  const int V = c.g.V;
  double2* d = nullptr;
  TSM_TRY(dalloc(&d, (size_t)2 * V * 12));
  const size_t off = (size_t)index * 3 * V * 8;
  int rc = TSM_OK;
  for (int w = 0; w < 2 && rc == TSM_OK; ++w) {
    pt_act_to_canon_kernel<<<dim3(grid1(V, NET_NT), 1), NET_NT, 0, c.stream>>>(V, 1, (w ? G.T : G.R) + off,
                                                                              d + (size_t)w * V * 12);
    rc = check_net_launch(c, "pt_act_to_canon_kernel");
  }
  if (rc == TSM_OK &&
      (cudaMemcpyAsync(r, d, (size_t)V * 12 * sizeof(double2), cudaMemcpyDeviceToHost, c.stream) != cudaSuccess ||
       cudaMemcpyAsync(t, d + (size_t)V * 12, (size_t)V * 12 * sizeof(double2), cudaMemcpyDeviceToHost, c.stream) !=
           cudaSuccess ||
       cudaStreamSynchronize(c.stream) != cudaSuccess))
    rc = nbad(TSM_ERR_CUDA, "pair copy failed");
  dfree(d);
  return rc;
}

namespace {

// one forward (+ loss, + backward when train) over pairs i0 .. i0+nb-1 of group g
int pair_step(Net& n, PairGroup& G, int i0, int nb, double* d_loss, bool train) {
  Ctx& c = *G.ctx;
  const size_t off = (size_t)i0 * 3 * c.g.V * 8;
  float* Y = nullptr;
  TSM_TRY(n.forward(c, G.R + off, nb, &Y));
  pt_loss_kernel<<<dim3(grid1(c.g.V, NET_NT), nb), NET_NT, 0, c.stream>>>(c.g, Y, G.T + off, G.den + i0, n.dA[1],
                                                                          d_loss);
  TSM_TRY(check_net_launch(c, "pt_loss_kernel"));
  if (train) TSM_TRY(n.backward(c, G.R + off, nb, n.dA[1], nullptr));
  return TSM_OK;
}

int loss_buffer(Net& n, int count) {
  if (count <= n.loss_cap) return TSM_OK;
  dfree(n.d_loss);
  TSM_TRY(dalloc(&n.d_loss, count));
  n.loss_cap = count;
  return TSM_OK;
}

}  // namespace

// Adam on the relative loss |net(r) - t|^2 / |t|^2 (even sites), minibatches
// of `batch` consecutive pairs, groups visited round-robin
extern "C" int tsm_net_train(tsm_net* h, const int* groups, int n_groups, int steps, int batch, double lr,
                             double* loss) {
  if (h == nullptr || groups == nullptr || n_groups < 1 || steps < 0 || batch < 1 || !(lr > 0.0))
    return nbad(TSM_ERR_ARG, "tsm_net_train: bad argument");
  Net& n = h->n;
  for (int i = 0; i < n_groups; ++i)
    if (groups[i] < 0 || groups[i] >= (int)n.groups.size()) return nbad(TSM_ERR_ARG, "unknown pair group");
  TSM_CUDA(cudaSetDevice(n.device));
  TSM_TRY(loss_buffer(n, std::max(steps, 1)));
  cudaStream_t s0 = n.groups[groups[0]].ctx->stream;
  TSM_CUDA(cudaMemsetAsync(n.d_loss, 0, std::max(steps, 1) * sizeof(double), s0));
  TSM_CUDA(cudaStreamSynchronize(s0));
  for (int g = 0; g < n_groups; ++g) TSM_TRY(zero_grads(n, n.groups[groups[g]].ctx->stream));
  for (int step = 0; step < steps; ++step) {
    PairGroup& G = n.groups[groups[step % n_groups]];
    const int nb = std::min(batch, G.n);
    const int chunks = G.n / nb;
    const int i0 = ((step / n_groups) % chunks) * nb;
    TSM_TRY(pair_step(n, G, i0, nb, n.d_loss + step, true));
    TSM_TRY(adam_step(n, G.ctx->stream, lr, 1.0 / nb));
    if (n_groups > 1) TSM_CUDA(cudaStreamSynchronize(G.ctx->stream));   // next step may use another stream
  }
  TSM_TRY(check_timeout(n, n.groups[groups[(steps + n_groups - 1) % n_groups]].ctx->stream));
  if (loss && steps > 0) {
    std::vector<double> hl(steps);
    TSM_CUDA(cudaMemcpy(hl.data(), n.d_loss, steps * sizeof(double), cudaMemcpyDeviceToHost));
    for (int st = 0; st < steps; ++st) {
      const PairGroup& G = n.groups[groups[st % n_groups]];
      loss[st] = hl[st] / std::min(batch, G.n);
    }
  }
  return TSM_OK;
}

// mean relative loss over all pairs of a group (no training)
extern "C" int tsm_net_loss(tsm_net* h, int group, double* loss) {
  if (h == nullptr || loss == nullptr) return nbad(TSM_ERR_ARG, "null argument");
  Net& n = h->n;
  if (group < 0 || group >= (int)n.groups.size()) return nbad(TSM_ERR_ARG, "unknown pair group");
  TSM_CUDA(cudaSetDevice(n.device));
  PairGroup& G = n.groups[group];
  TSM_TRY(loss_buffer(n, 1));
  TSM_CUDA(cudaMemsetAsync(n.d_loss, 0, sizeof(double), G.ctx->stream));
  const int nb = std::min(G.n, 16);
  for (int i0 = 0; i0 < G.n; i0 += nb) TSM_TRY(pair_step(n, G, i0, std::min(nb, G.n - i0), n.d_loss, false));
  TSM_TRY(check_timeout(n, G.ctx->stream));
  double s = 0.0;
  TSM_CUDA(cudaMemcpy(&s, n.d_loss, sizeof(double), cudaMemcpyDeviceToHost));
  *loss = s / G.n;
  return TSM_OK;
}

extern "C" int tsm_set_precond(tsm_ctx* ch, tsm_net* h) {
  if (ch == nullptr) return nbad(TSM_ERR_ARG, "null context");
  if (h != nullptr && h->n.device != ch->c.device)
    return nbad(TSM_ERR_ARG, "network and context live on different devices");
  ch->c.net = h ? &h->n : nullptr;
  return TSM_OK;
}
