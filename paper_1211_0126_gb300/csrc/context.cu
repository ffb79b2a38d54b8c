// context.cu -- workspace, error reporting and instrumentation of a context.
#include <cstdarg>
#include <cstdio>

#include "context.h"

namespace tsm {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

const char* last_error() { return g_err; }

size_t field_bytes(int prec, int vh) {
  switch (prec) {
    case TSM_F64: return (size_t)vh * 12 * sizeof(double2);
    case TSM_F32: return (size_t)vh * 6 * sizeof(float4);
    default: return (size_t)vh * 3 * sizeof(uint4);
  }
}

double spinor_site_bytes(int prec) {
  switch (prec) {
    case TSM_F64: return 24.0 * 8;
    case TSM_F32: return 24.0 * 4;
    default: return 24.0 * 2;
  }
}

double link_site_bytes(int prec) {
  switch (prec) {
    case TSM_F64: return 8.0 * 18 * 8;   // FP64 links keep all three rows
    case TSM_F32: return 8.0 * 12 * 4;
    default: return 8.0 * 12 * 2;
  }
}

int check_launch(Ctx& c, const char* what) {
  (void)c;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("launch of %s failed: %s", what, cudaGetErrorString(e));
    return TSM_ERR_CUDA;
  }
  return TSM_OK;
}

int Ctx::buffer(const std::string& base_name, size_t bytes, void** out) {
  const std::string name = ws_prefix + base_name;
  auto it = ws.find(name);
  if (it != ws.end() && it->second.second >= bytes) {
    *out = it->second.first;
    return TSM_OK;
  }
  if (capturing) {
    set_error("workspace '%s' was not reserved before graph capture", name.c_str());
    return TSM_ERR_ARG;
  }
  if (it != ws.end()) {
    TSM_CUDA(cudaStreamSynchronize(stream));
    TSM_CUDA(cudaFree(it->second.first));
    ws.erase(it);
  }
  void* p = nullptr;
  if (bytes > 0) TSM_CUDA(cudaMalloc(&p, bytes));
  ws[name] = {p, bytes};
  *out = p;
  return TSM_OK;
}

int Ctx::field(const std::string& name, int prec, PField* f, int nrhs) {
  return buffer(name + "#" + std::to_string(prec), field_bytes(prec, sstride) * (size_t)(nrhs > 0 ? nrhs : 1), &f->p);
}

int Ctx::harvest_events() {
  if (ev_pending.empty()) return TSM_OK;
  TSM_CUDA(cudaStreamSynchronize(stream));
  for (auto& r : ev_pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      prof_ms[r.kind] += ms;
      prof_cnt[r.kind] += 1;
      prof_bytes[r.kind] += r.bytes;
    } else {
      (void)cudaGetLastError();   // an untimed pair: leave no error behind for the caller
    }
    ev_free.push_back(r);
  }
  ev_pending.clear();
  return TSM_OK;
}

void Ctx::free_all() {
  cudaStreamSynchronize(stream);
  for (auto& kv : ws) cudaFree(kv.second.first);
  ws.clear();
  for (int k = 0; k < 4; ++k) {
    if (links[k]) cudaFree(links[k]);
    links[k] = nullptr;
  }
  if (red.partials) cudaFree(red.partials);
  if (red.counter) cudaFree(red.counter);
  if (red_branch.partials) cudaFree(red_branch.partials);
  if (red_branch.counter) cudaFree(red_branch.counter);
  red_branch = RedSlot{};
  red = RedSlot{};
  if (states) cudaFree(states);
  if (h_states) cudaFreeHost(h_states);
  if (d_lists) cudaFree(d_lists);
  if (d_guard) cudaFree(d_guard);
  d_guard = nullptr;
  if (h_lists) cudaFreeHost(h_lists);
  states = nullptr;
  h_states = nullptr;
  d_lists = nullptr;
  h_lists = nullptr;
  for (auto& r : ev_free) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto& r : ev_pending) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  ev_free.clear();
  ev_pending.clear();
}

}  // namespace tsm
