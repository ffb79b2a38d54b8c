// context.h -- host-side state of a library context and the launch helpers
// shared by the solver and the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <map>
#include <string>
#include <vector>

#include "tsm.h"
#include "common.cuh"
#include "dslash.cuh"

namespace tsm {

void set_error(const char* fmt, ...);

#define TSM_CUDA(call)                                                               \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) {                                                         \
      ::tsm::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),       \
                       __FILE__, __LINE__);                                          \
      return TSM_ERR_CUDA;                                                           \
    }                                                                                \
  } while (0)

#define TSM_TRY(expr)          \
  do {                         \
    int s_ = (expr);           \
    if (s_ != TSM_OK) return s_; \
  } while (0)

// one parity field of any storage (pointer to chunk 0; chunk stride = Ctx::sstride)
struct PField {
  void* p = nullptr;
  template <class S> typename S::schunk* as() const { return static_cast<typename S::schunk*>(p); }
};

// even + odd parity fields
struct EOField {
  PField e, o;
  PField& par(int parity) { return parity ? o : e; }
};

enum HopKind { PK_HOP = 0, PK_HOP_XPAY = 1, PK_HOP_DAG = 2, PK_HOP_UPDATE = 3 };
// profile buckets after the 16 hop buckets: local contraction passes (kernel +
// fixed-order reduction, every estimator), derivative-insertion passes, the
// all-momenta FFT projection (densities, the transform, running moments), the Wilson
// application of the generalised one-end estimator
enum ProfContract { PB_CONTRACT = 16, PB_DERIV = 17, PB_FFT = 18, PB_WILSON = 19 };

struct Net;

struct Ctx {
  int device = 0;
  Net* net = nullptr;    // learned preconditioner used by solves with tm_stop.precond (not owned)
  cudaStream_t stream = nullptr;
  bool has_gauge = false;
  tm_lattice lat{};
  Geom g{};
  int sstride = 0;       // chunk stride of parity fields (= Vh)
  int lstride = 0;       // chunk stride of link fields (= Vh)
  void* links[4] = {nullptr, nullptr, nullptr, nullptr};   // F64, F32, BF16, F16: [2][4][LN][lstride]
  std::map<std::string, std::pair<void*, size_t>> ws;      // named device workspace
  RedSlot red{};
  size_t red_cap = 0;
  CGState* states = nullptr;    // device, kMaxStates
  CGState* h_states = nullptr;  // pinned mirror
  static constexpr int kMaxStates = 2048;  // last 4 reserved for auxiliary reductions
  static constexpr int kMaxBatch = 64;     // right-hand sides per batched solve
  static constexpr int kMaxGuards = 256;   // while-loop iteration guards of one captured graph
  int* d_lists = nullptr;       // device: 3 lists of kMaxBatch right-hand-side indices
  int* h_lists = nullptr;       // pinned staging of the lists
  int* d_guard = nullptr;       // device iteration counters of captured while-loops
  int batch_cap = 1;            // batch width the solver workspace is laid out for
  // graph capture: solves become graph while-loops on `stream`, their bodies
  // are captured on `body_stream`, states are taken from `next_state` onwards
  bool capturing = false;
  cudaStream_t body_stream = nullptr;
  // second branch of a captured run (the LP set beside the HP set): its own
  // stream, workspace (names prefixed by ws_prefix) and reduction slots
  cudaStream_t branch_stream = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  std::string ws_prefix;
  RedSlot red_branch{};
  size_t red_branch_cap = 0;
  int next_state = 0;
  int next_guard = 0;
  std::vector<int> guard_body_launches;   // kernels in the body of each captured while-loop
  std::vector<std::pair<int, int>> cap_lp, cap_hp;   // (first state, count) of captured solves
  std::map<std::string, int> tuned_batch;            // autotuner cache: lattice + tier -> batch width
  std::map<std::string, int> tuned_rpb;              // autotuner cache: lattice + tier -> block shape index
  // sources per link-sharing block of the 16-bit and FP32 stencils, per tier id
  // (2, 4 or 8), and the register budget of the 4-source blocks (80 or 96); the
  // autotuner sets them, the results do not depend on them
  int tile_rpb[4] = {LT_RHS, LT_RHS, LT_RHS, LT_RHS};
  int tile_regs[4] = {LT_REGS, LT_REGS, LT_REGS, LT_REGS};   // register budget of the 4-source tiles
  // instrumentation
  bool profile = false;
  struct EvRec {
    cudaEvent_t a, b;
    int kind;
    double bytes;
  };
  std::vector<EvRec> ev_free, ev_pending;
  // 4 storage tiers x 4 hop kinds, then the contraction kinds (ProfContract)
  static constexpr int kProfBuckets = 24;
  double prof_ms[kProfBuckets] = {};
  long long prof_cnt[kProfBuckets] = {};
  double prof_bytes[kProfBuckets] = {};
  bool prof_this_launch = false;   // solver sets it for the instrumented iteration
  // single-source operator applications outside the solvers (tm_dslash): the
  // 16-bit tiers use the one-thread-per-site stencil instead of link sharing
  bool hop_per_site = false;
  long long launches = 0;

  // device buffer by name, (re)allocated when too small; contents undefined
  int buffer(const std::string& name, size_t bytes, void** out);
  template <class S> const typename S::lchunk* links_of(int parity) const {
    return static_cast<const typename S::lchunk*>(links[S::id]) + (size_t)parity * 4 * S::LN * lstride;
  }
  int field(const std::string& name, int prec, PField* f, int nrhs = 1);   // nrhs parity fields of tier prec
  int harvest_events();                                        // sync + accumulate profile times
  void free_all();
};

size_t field_bytes(int prec, int vh);

// field of right-hand side `rhs` inside a batch of contiguous parity fields
inline PField field_at(const PField& f, int prec, int vh, int rhs) {
  return PField{static_cast<char*>(f.p) + field_bytes(prec, vh) * (size_t)rhs};
}
inline EOField eo_at(const EOField& f, int prec, int vh, int rhs) {
  return EOField{field_at(f.e, prec, vh, rhs), field_at(f.o, prec, vh, rhs)};
}

// Twist factors (diagonal in the chiral basis)
inline Twist twist_one() { return Twist{{1.0, 1.0}, {0.0, 0.0}}; }
inline Twist twist_scale(double s) { return Twist{{s, s}, {0.0, 0.0}}; }
// A(m) = 1 + 2 i kappa m gamma5
inline Twist twist_A(double kappa, double m) {
  return Twist{{1.0, 1.0}, {2.0 * kappa * m, -2.0 * kappa * m}};
}
// A(m)^-1 = (1 - 2 i kappa m gamma5) / (1 + 4 kappa^2 m^2)
inline Twist twist_Ainv(double kappa, double m) {
  const double d = 1.0 + 4.0 * kappa * kappa * m * m;
  return Twist{{1.0 / d, 1.0 / d}, {-2.0 * kappa * m / d, 2.0 * kappa * m / d}};
}
// the product of two twists (they commute: both are diagonal)
inline Twist twist_mul(const Twist& a, const Twist& b) {
  Twist t;
  for (int q = 0; q < 2; ++q) {
    t.re[q] = a.re[q] * b.re[q] - a.im[q] * b.im[q];
    t.im[q] = a.re[q] * b.im[q] + a.im[q] * b.re[q];
  }
  return t;
}

// ---- launch helpers (instantiated per storage type in ops_*.cu).  Batched
// helpers take nrhs right-hand sides stored as contiguous parity fields (the
// grid's x dimension), optionally through a device list `active` of the
// right-hand sides still iterating.
template <class S> int launch_hop(Ctx& c, const HopArgs<S>& a, int dag, int mode, int prof_kind, int nrhs = 1);
template <class S, class SA> int launch_cg_update(Ctx& c, const CGUpdArgs<S, SA>& a, int nrhs);
template <class S, class SA>
int launch_cg_p(Ctx& c, const PField& r, const PField& p, CGState* st, const int* active, int nrhs);
template <class S> int launch_pack(Ctx& c, int parity, const double* canon, const PField& out);
template <class S> int launch_unpack(Ctx& c, int parity, const PField& in, double* canon);
template <class S>
int launch_noise(Ctx& c, int parity, const NoiseSpec& n, uint32_t source0, const PField& out, int nrhs = 1);
template <class S>
int launch_twist(Ctx& c, const Twist& f, const PField& in, const PField& out, const CGState* st,
                 const int* active = nullptr, int nrhs = 1);
template <class S>
int launch_norm(Ctx& c, const PField& v, CGState* st, int post, const int* active = nullptr, int nrhs = 1);
template <class Si, class So>
int launch_convert(Ctx& c, const PField& in, const PField& out, const int* active = nullptr, int nrhs = 1);

// runtime dispatch on a tier id (0 F64, 1 F32, 2 BF16, 3 F16):
// f receives an empty tag object of the storage type
template <class F>
int dispatch_prec(int prec, F&& f) {
  switch (prec) {
    case TSM_F64: return f(F64{});
    case TSM_F32: return f(F32{});
    case TSM_BF16: return f(BF16{});
    case TSM_F16: return f(F16{});
    default: return TSM_ERR_ARG;
  }
}

// algorithmic bytes of one hop-kernel launch for storage S (per output site:
// 8 links x 12 reals, one input spinor, one output spinor, plus the extra
// streams of the fused epilogues) -- used only for instrumentation
double spinor_site_bytes(int prec);
double link_site_bytes(int prec);   // 8 links x 12 reals

// records the CUDA-event time of the launches it brackets when instrumentation
// is on for this launch (c.profile && c.prof_this_launch); bytes = algorithmic bytes
struct TimedLaunch {
  Ctx& c;
  Ctx::EvRec rec{};
  bool on = false;
  // any_launch: time it whenever instrumentation is on (contraction buckets)
  TimedLaunch(Ctx& cc, int kind, double bytes, bool any_launch = false) : c(cc) {
    // under stream capture an event record becomes a dependency, not a time
    if (!c.profile || c.capturing || !(c.prof_this_launch || any_launch)) return;
    if (c.ev_free.empty()) {
      Ctx::EvRec r{};
      if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) return;
      c.ev_free.push_back(r);
    }
    rec = c.ev_free.back();
    c.ev_free.pop_back();
    rec.kind = kind;
    rec.bytes = bytes;
    on = (cudaEventRecord(rec.a, c.stream) == cudaSuccess);
    if (!on) c.ev_free.push_back(rec);
  }
  void done() {
    if (!on) return;
    if (cudaEventRecord(rec.b, c.stream) == cudaSuccess) c.ev_pending.push_back(rec);
    else c.ev_free.push_back(rec);
    on = false;
  }
};

int check_launch(Ctx& c, const char* what);

}  // namespace tsm

struct tsm_ctx {
  tsm::Ctx c;
};
