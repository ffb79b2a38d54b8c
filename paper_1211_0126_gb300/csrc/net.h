// net.h -- the learned LP preconditioner: a stack of gauge-covariant
// parallel-transport layers with tensor-core channel mixing (kernels in
// ptnet.cuh, GEMM in umma.cuh), its training state and its use inside
// flexible GMRES.
#pragma once

#include <cuda_bf16.h>

#include <vector>

#include "context.h"

namespace tsm {

int launch_umma_gemm_ex(cudaStream_t stream, const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb,
                        float* C, int ldc, int M, int N, int K, int beta, int splits, int* error,
                        int* used_splits);
int launch_umma_gemm(cudaStream_t stream, const __nv_bfloat16* A, const __nv_bfloat16* B, float* C, int M, int N,
                     int K, int ldc, int beta, int* error);

struct NetLayer {
  int cin = 0, cout = 0;
  float *wr = nullptr, *wi = nullptr;      // FP32 master weights [4 cout][36 cin]
  float *gr = nullptr, *gi = nullptr;      // gradient accumulators
  float *mr = nullptr, *vr = nullptr, *mi = nullptr, *vi = nullptr;   // Adam moments
  __nv_bfloat16 *B = nullptr, *Bt = nullptr;   // packed block weights [8 cout][72 cin] and transpose
  int n4() const { return 4 * cout; }
  int k36() const { return 36 * cin; }
};

// training pairs (r, Dhat^-1 r) of one gauge field, stored as one-channel
// activations (odd sites zero)
struct PairGroup {
  Ctx* ctx = nullptr;
  int n = 0;
  float* R = nullptr;     // [n][3V][8]
  float* T = nullptr;     // [n][3V][8]
  double* den = nullptr;  // [n]: sum over even sites of |T|^2
};

struct Net {
  int device = 0;
  std::vector<NetLayer> layers;
  std::vector<PairGroup> groups;
  int adam_t = 0;
  bool packed = false;     // B / Bt up to date with the master weights
  int* d_err = nullptr;    // tensor-core wait timeout flag
  double* d_loss = nullptr;
  int loss_cap = 0;
  // activation workspace for (V, nb)
  int ws_V = 0, ws_nb = 0;
  std::vector<float*> acts;           // L + 1 activations
  __nv_bfloat16* Z = nullptr;         // gathered input [M][72 cmax]
  __nv_bfloat16* Zt = nullptr;        // its transpose
  float* dZ = nullptr;                // [M][72 cmax]
  float* dA[2] = {nullptr, nullptr};  // activation gradients [M][8 cmax]
  __nv_bfloat16* dYb = nullptr;       // [M][8 cmax]
  __nv_bfloat16* dYt = nullptr;       // [8 cmax][M]
  float* part = nullptr;              // split-K partials of the weight gradient
  size_t part_cap = 0;
  int cmax() const;
  int reserve(int V, int nb);
  int pack(cudaStream_t s);
  // forward pass of nb samples whose input activations are at X0 (one
  // channel); activations kept in acts[1..L]; returns the output activation
  int forward(Ctx& c, const float* X0, int nb, float** out);
  // backward pass given the output gradient dY (acts[0] = X0 of the forward);
  // accumulates weight gradients, writes the input gradient to dX0 if non-null
  int backward(Ctx& c, const float* X0, int nb, const float* dY, float* dX0);
  void free_all();
};

// Apply the preconditioner to nrhs even-site FP32 parity fields (M out = net(in)).
int net_apply_even(Ctx& c, Net& n, const PField& in, const PField& out, int nrhs);

// Flexible GMRES on Dhat x = bhat with the network as right preconditioner
// (plain CG on the same tier when it breaks down); fields as in solve_batch.
struct SolveResult;
int fgmres_batch(Ctx& c, const tm_stop& stop, int nrhs, EOField b, EOField s, SolveResult* res);

}  // namespace tsm

struct tsm_net {
  tsm::Net n;
};
