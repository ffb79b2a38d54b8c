// noalloc.cu -- a loop contraction that allocates no memory.
//
// Some callers cannot allocate device memory at the point where they need a
// contraction: code running under a foreign memory manager that owns the
// whole device (a framework's caching allocator or a fixed-size arena),
// real-time or signal-handling paths where cudaMalloc's implicit device
// synchronisation and unbounded latency are not acceptable, or callers that
// hold no tsm_ctx at all.  tsm_contract_noalloc serves them: the caller passes
// the solution and the output buffer (device memory it already owns) and the
// function uses only the fixed scratch array below, which exists once per
// device for as long as the library stays loaded.
//
// Scratch layout (double2 entries): [phase tables n_q x (Lx+Ly+Lz)]
// [block partial sums T x nsplit x (n_gamma * n_q)].  Every entry the kernels
// read is written earlier in the same call, so nothing has to be cleared
// between calls.  All calls on a device share the one array: two calls whose
// kernels overlap on the GPU (different streams without ordering, or several
// host threads) race on it and must be serialised by the caller.
//
// The host only knows the array by its symbol; its device address is looked
// up with cudaGetSymbolAddress on every call, with the caller's device
// current.  The lookup allocates nothing, and a fresh one per call stays
// right after a device reset, when the module is loaded again and the array
// may sit at another address.
#include <mutex>

#include "contract.h"

namespace tsm {

// capacity of the scratch array: 1 MiB per device
constexpr int kNoallocEntries = 65536;
constexpr int kNoallocNT = 128;

static __device__ __align__(256) double2 g_noalloc_scratch[kNoallocEntries];

// One block sums a contiguous chunk of the full-lattice sites of timeslice
// blockIdx.y; the canonical spinor is read directly (no repacking, hence no
// workspace).  FP64 throughout, like tsm_contract with TSM_F64.
struct NoallocArgs {
  Geom g;
  NoiseSpec noise;
  uint32_t source;
  const double2* s;     // canonical [V][12]
  GammaTab gam;
  int nq;
  const double2* phx;
  const double2* phy;
  const double2* phz;
  double2* partial;     // [T][nsplit][nout]
  int nsplit;
};

static __global__ void __launch_bounds__(kNoallocNT) noalloc_contract_kernel(const NoallocArgs a) {
  __shared__ cx<double> Gs[kNoallocNT][CT_MAXG + 1];
  __shared__ cx<double> Ps[kNoallocNT][CT_MAXQ + 1];
  const int t = blockIdx.y;
  const int vs = a.g.L[0] * a.g.L[1] * a.g.L[2];
  const int per = (vs + a.nsplit - 1) / a.nsplit;
  const int lo = blockIdx.x * per, hi = min(vs, lo + per);
  const int ng = a.gam.n, nq = a.nq, nout = ng * nq;
  // running (g, q) sums of this block, one output per thread (nout <= 256)
  cx<double> acc0 = {0, 0}, acc1 = {0, 0};
  for (int base = lo; base < hi; base += kNoallocNT) {
    const int local = base + threadIdx.x;
    if (local < hi) {
      const int lex = t * vs + local;
      int r = lex;
      const int x = r % a.g.L[0];
      r /= a.g.L[0];
      const int y = r % a.g.L[1];
      r /= a.g.L[1];
      const int z = r % a.g.L[2];
      cx<double> eta[12], s[12];
      noise_site<double>(a.noise, (uint32_t)lex, a.source, eta);
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        const double2 v = a.s[(size_t)lex * 12 + k];
        s[k] = {v.x, v.y};
      }
      cx<double> S[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
          S[i][j] = cjmul(eta[3 * i], s[3 * j]) + cjmul(eta[3 * i + 1], s[3 * j + 1]) +
                    cjmul(eta[3 * i + 2], s[3 * j + 2]);
      for (int k = 0; k < ng; ++k) {
        cx<double> v = {0, 0};
#pragma unroll
        for (int row = 0; row < 4; ++row) {
          const int col = a.gam.col[k][row];
          cx<double> sv;
          switch (col) {
            case 0: sv = S[row][0]; break;
            case 1: sv = S[row][1]; break;
            case 2: sv = S[row][2]; break;
            default: sv = S[row][3]; break;
          }
          v = v + times_ipow(sv, a.gam.ph[k][row]);
        }
        Gs[threadIdx.x][k] = v;
      }
      for (int q = 0; q < nq; ++q) {
        const double2 ex = a.phx[q * a.g.L[0] + x];
        const double2 ey = a.phy[q * a.g.L[1] + y];
        const double2 ez = a.phz[q * a.g.L[2] + z];
        Ps[threadIdx.x][q] = (cx<double>{ex.x, ex.y} * cx<double>{ey.x, ey.y}) * cx<double>{ez.x, ez.y};
      }
    } else {
      for (int k = 0; k < ng; ++k) Gs[threadIdx.x][k] = {0, 0};
      for (int q = 0; q < nq; ++q) Ps[threadIdx.x][q] = {0, 0};
    }
    __syncthreads();
    for (int k = threadIdx.x, slot = 0; k < nout; k += kNoallocNT, ++slot) {
      const int gi = k % ng, q = k / ng;
      cx<double> sum = {0, 0};
      for (int s2 = 0; s2 < kNoallocNT; ++s2) sum = sum + Ps[s2][q] * Gs[s2][gi];
      if (slot == 0) acc0 = acc0 + sum;
      else acc1 = acc1 + sum;
    }
    __syncthreads();
  }
  double2* dst = a.partial + ((size_t)t * a.nsplit + blockIdx.x) * nout;
  for (int k = threadIdx.x, slot = 0; k < nout; k += kNoallocNT, ++slot) {
    const cx<double> v = slot == 0 ? acc0 : acc1;
    dst[k] = make_double2(v.re, v.im);
  }
}

// out[(g * nq + q) * T + t] = sum over the block partials of timeslice t, in block order
static __global__ void noalloc_reduce_kernel(const double2* __restrict__ partial, int T, int nsplit, int ng, int nq,
                                             double2* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int nout = ng * nq;
  if (k >= nout * T) return;
  const int t = k % T, gq = k / T;
  double re = 0.0, im = 0.0;
  for (int b = 0; b < nsplit; ++b) {
    const double2 v = partial[((size_t)t * nsplit + b) * nout + gq];
    re += v.x;
    im += v.y;
  }
  const int gi = gq % ng, q = gq / ng;
  out[((size_t)gi * nq + q) * T + t] = make_double2(re, im);
}

namespace {
std::mutex g_noalloc_mutex;
// host staging of the phase tables (a fixed host array: no heap allocation)
double2 g_noalloc_phase[CT_MAXQ * 3 * 1024];
}  // namespace

}  // namespace tsm

using namespace tsm;

extern "C" int tsm_contract_noalloc(const tm_lattice* lat, uint64_t seed, int kind, uint32_t source,
                                    const double* s_dev, const int* gammas, int n_gamma, const int* moms, int n_q,
                                    double* out_dev, void* cuda_stream) {
  if (lat == nullptr || s_dev == nullptr || out_dev == nullptr || gammas == nullptr || moms == nullptr) {
    set_error("tsm_contract_noalloc: null argument");
    return TSM_ERR_ARG;
  }
  if (kind != 4 && kind != 2) {
    set_error("tsm_contract_noalloc: noise kind must be 4 or 2");
    return TSM_ERR_ARG;
  }
  long long V = 1;
  for (int k = 0; k < 4; ++k) {
    if (lat->L[k] < 2 || (lat->L[k] & 1)) {
      set_error("tsm_contract_noalloc: every extent must be even and >= 2");
      return TSM_ERR_DIMS;
    }
    V *= lat->L[k];
  }
  if (V >= (1ll << 31)) {
    set_error("tsm_contract_noalloc: lattice too large for 32-bit site indexing");
    return TSM_ERR_DIMS;
  }
  if (n_gamma < 1 || n_gamma > CT_MAXG || n_q < 1 || n_q > CT_MAXQ) {
    set_error("tsm_contract_noalloc: needs 1 <= n_gamma <= %d and 1 <= n_q <= %d (got %d, %d)", CT_MAXG, CT_MAXQ,
              n_gamma, n_q);
    return TSM_ERR_TOO_LARGE;
  }
  const int T = lat->L[3];
  const int lsum = lat->L[0] + lat->L[1] + lat->L[2];
  const int n_phase = n_q * lsum;
  if (lsum > 3 * 1024) {
    set_error("tsm_contract_noalloc: Lx + Ly + Lz = %d above the limit 3072", lsum);
    return TSM_ERR_TOO_LARGE;
  }
  const int nout = n_gamma * n_q;
  // enough blocks to cover the SMs, within the scratch capacity
  int nsplit = (608 + T - 1) / T;
  const int vs = lat->L[0] * lat->L[1] * lat->L[2];
  if (nsplit > vs / kNoallocNT) nsplit = vs / kNoallocNT > 0 ? vs / kNoallocNT : 1;
  while (nsplit > 1 && (long long)n_phase + (long long)T * nsplit * nout > kNoallocEntries) --nsplit;
  if ((long long)n_phase + (long long)T * nsplit * nout > kNoallocEntries) {
    set_error("tsm_contract_noalloc: needs %lld scratch entries, capacity is %d (1 MiB)",
              (long long)n_phase + (long long)T * nout, kNoallocEntries);
    return TSM_ERR_TOO_LARGE;
  }
  GammaTab gt{};
  int rc = make_gamma_tab(gammas, n_gamma, &gt);
  if (rc != TSM_OK) return rc;
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  // device address of the scratch array on the current device (the symbol
  // itself is a host-side stand-in that no kernel may be given)
  void* sym = nullptr;
  const cudaError_t se = cudaGetSymbolAddress(&sym, g_noalloc_scratch);
  if (se != cudaSuccess || sym == nullptr) {
    set_error("tsm_contract_noalloc: cudaGetSymbolAddress of the scratch array failed: %s", cudaGetErrorString(se));
    return TSM_ERR_CUDA;
  }
  double2* scratch = static_cast<double2*>(sym);
  const double twopi = 2.0 * std::acos(-1.0);
  int off = 0;
  for (int ax = 0; ax < 3; ++ax)
    for (int q = 0; q < n_q; ++q)
      for (int x = 0; x < lat->L[ax]; ++x) {
        long long nx = (long long)moms[3 * q + ax] * x;
        nx %= lat->L[ax];
        if (nx < 0) nx += lat->L[ax];
        const double ang = twopi * (double)nx / (double)lat->L[ax];
        g_noalloc_phase[off++] = make_double2(std::cos(ang), std::sin(ang));
      }
  // pageable source: the copy has consumed the host table when the call returns
  TSM_CUDA(cudaMemcpyAsync(scratch, g_noalloc_phase, (size_t)n_phase * sizeof(double2), cudaMemcpyHostToDevice,
                           stream));
  NoallocArgs a{};
  a.g = make_geom(lat->L, lat->t_antiperiodic);
  a.noise = make_noise(seed, kind);
  a.source = source;
  a.s = reinterpret_cast<const double2*>(s_dev);
  a.gam = gt;
  a.nq = n_q;
  a.phx = scratch;
  a.phy = scratch + (size_t)n_q * lat->L[0];
  a.phz = a.phy + (size_t)n_q * lat->L[1];
  a.partial = scratch + n_phase;
  a.nsplit = nsplit;
  noalloc_contract_kernel<<<dim3(nsplit, T), kNoallocNT, 0, stream>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("tsm_contract_noalloc: contraction launch failed: %s", cudaGetErrorString(e));
    return TSM_ERR_CUDA;
  }
  const int nred = nout * T;
  noalloc_reduce_kernel<<<(nred + 127) / 128, 128, 0, stream>>>(a.partial, T, nsplit, n_gamma, n_q,
                                                                reinterpret_cast<double2*>(out_dev));
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("tsm_contract_noalloc: reduction launch failed: %s", cudaGetErrorString(e));
    return TSM_ERR_CUDA;
  }
  return TSM_OK;
}
