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

struct Ctx {
  int device = 0;
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
  static constexpr int kMaxStates = 64;
  // instrumentation
  bool profile = false;
  struct EvRec {
    cudaEvent_t a, b;
    int kind;
    double bytes;
  };
  std::vector<EvRec> ev_free, ev_pending;
  double prof_ms[4] = {0, 0, 0, 0};
  long long prof_cnt[4] = {0, 0, 0, 0};
  double prof_bytes[4] = {0, 0, 0, 0};
  bool prof_this_launch = false;   // solver sets it for the instrumented iteration
  long long launches = 0;

  // device buffer by name, (re)allocated when too small; contents undefined
  int buffer(const std::string& name, size_t bytes, void** out);
  template <class S> const typename S::lchunk* links_of(int parity) const {
    return static_cast<const typename S::lchunk*>(links[S::id]) + (size_t)parity * 4 * S::LN * lstride;
  }
  int field(const std::string& name, int prec, PField* f);    // one parity field of tier prec
  int harvest_events();                                        // sync + accumulate profile times
  void free_all();
};

size_t field_bytes(int prec, int vh);

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

// ---- launch helpers (instantiated per storage type in ops_*.cu)
template <class S> int launch_hop(Ctx& c, const HopArgs<S>& a, int dag, int mode, int prof_kind);
template <class S, class SA> int launch_cg_update(Ctx& c, const CGUpdArgs<S, SA>& a);
template <class S, class SA> int launch_cg_p(Ctx& c, const PField& r, const PField& p, CGState* st);
template <class S> int launch_pack(Ctx& c, int parity, const double* canon, const PField& out);
template <class S> int launch_unpack(Ctx& c, int parity, const PField& in, double* canon);
template <class S> int launch_noise(Ctx& c, int parity, const NoiseSpec& n, uint32_t source, const PField& out);
template <class S> int launch_twist(Ctx& c, const Twist& f, const PField& in, const PField& out, const CGState* st);
template <class S> int launch_norm(Ctx& c, const PField& v, CGState* st, int post);
template <class Si, class So> int launch_convert(Ctx& c, const PField& in, const PField& out);

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

int check_launch(Ctx& c, const char* what);

}  // namespace tsm

struct tsm_ctx {
  tsm::Ctx c;
};
