// Per-stage timing with CUDA events, NVTX ranges and a count of kernel
// launches.
//
// When enabled, each stage of compress / decompress records a pair of events
// on the caller's stream; elapsed times are folded in when they are read
// (qoz_profile_read synchronises on the recorded events).  Every stage also
// opens an NVTX range named after it (a no-op unless a tool is attached), so
// a timeline shows the library's stages.  The launch counter is always on:
// every kernel launch of the library increments it.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <atomic>
#include <mutex>
#include <vector>

#include "../../include/qoz.h"
#include "qoz_host.h"
#include "qoz_internal.h"

namespace qoz {
namespace {

struct Pending {
  int stage;
  cudaEvent_t a, b;
};

std::mutex g_mu;
std::atomic<bool> g_on{false};
std::atomic<unsigned> g_mask{0xffffffffu};
std::atomic<long long> g_launches{0};
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_free;
double g_ms[QOZ_PROF_STAGES];
long long g_calls[QOZ_PROF_STAGES];

cudaEvent_t take_event() {
  if (!g_free.empty()) {
    cudaEvent_t e = g_free.back();
    g_free.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

void fold_pending_locked() {
  for (const Pending& p : g_pending) {
    float ms = 0.0f;
    if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      g_ms[p.stage] += ms;
      g_calls[p.stage] += 1;
    }
    g_free.push_back(p.a);
    g_free.push_back(p.b);
  }
  g_pending.clear();
}

}  // namespace

void note_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// NVTX range names of the stages (the host-side span of each stage).
const char* stage_name(int stage) {
  static const char* const level[] = {"qoz level 1", "qoz level 2", "qoz level 3", "qoz level 4",
                                      "qoz level 5", "qoz level 6", "qoz level 7", "qoz level 8"};
  static const char* const dlevel[] = {"qoz decode level 1", "qoz decode level 2",
                                       "qoz decode level 3", "qoz decode level 4",
                                       "qoz decode level 5", "qoz decode level 6",
                                       "qoz decode level 7", "qoz decode level 8"};
  if (stage == QOZ_STAGE_RANGE) return "qoz value range";
  if (stage == QOZ_STAGE_SETUP) return "qoz bounds + anchors";
  if (stage > QOZ_STAGE_LEVEL && stage <= QOZ_STAGE_LEVEL + 8) return level[stage - QOZ_STAGE_LEVEL - 1];
  if (stage == QOZ_STAGE_HIST) return "qoz histogram";
  if (stage == QOZ_STAGE_FINAL) return "qoz unpredictable list";
  if (stage > QOZ_STAGE_DLEVEL && stage <= QOZ_STAGE_DLEVEL + 8)
    return dlevel[stage - QOZ_STAGE_DLEVEL - 1];
  if (stage == QOZ_STAGE_METRICS) return "qoz metrics";
  if (stage == QOZ_STAGE_TUNE) return "qoz tuner trials";
  return "qoz stage";
}

ProfScope::ProfScope(int stage, cudaStream_t s) : stage_(stage), s_(s), a_(nullptr) {
  nvtxRangePushA(stage_name(stage));
  if (!g_on.load(std::memory_order_relaxed) || stage < 0 || stage >= QOZ_PROF_STAGES) return;
  if (!((g_mask.load(std::memory_order_relaxed) >> stage) & 1u)) return;
  std::lock_guard<std::mutex> lk(g_mu);
  a_ = take_event();
  if (a_ && cudaEventRecord(a_, s_) != cudaSuccess) {
    g_free.push_back(a_);
    a_ = nullptr;
  }
}

ProfScope::~ProfScope() {
  nvtxRangePop();
  if (!a_) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEvent_t b = take_event();
  if (!b || cudaEventRecord(b, s_) != cudaSuccess) {
    g_free.push_back(a_);
    if (b) g_free.push_back(b);
    return;
  }
  g_pending.push_back({stage_, a_, b});
}

}  // namespace qoz

using namespace qoz;

extern "C" {

qoz_status qoz_profile_enable(int32_t enable) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_on.store(enable != 0);
  return QOZ_OK;
}

qoz_status qoz_debug_bounds(uint64_t* first_bad, int32_t reset) {
  if (!first_bad) return fail(QOZ_EINVAL, "NULL argument");
#ifdef QOZ_DEBUG_BOUNDS
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "bounds record");
  const unsigned long long w[4] = {bounds_take_level(reset != 0),
                                   bounds_take_level_batch(reset != 0),
                                   bounds_take_tune(reset != 0), bounds_take_entropy(reset != 0)};
  *first_bad = 0;
  for (unsigned long long v : w)
    if (v && !*first_bad) *first_bad = v;
  return QOZ_OK;
#else
  *first_bad = 0;
  (void)reset;
  return fail(QOZ_EUNSUPPORTED, "not the bounds-checking build (QOZ_DEBUG_BOUNDS)");
#endif
}

qoz_status qoz_profile_stages(uint32_t mask) {
  g_mask.store(mask);
  return QOZ_OK;
}

qoz_status qoz_profile_read(qoz_stage_times* out, int32_t reset) {
  if (!out) return fail(QOZ_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(g_mu);
  fold_pending_locked();
  for (int i = 0; i < QOZ_PROF_STAGES; ++i) {
    out->ms[i] = g_ms[i];
    out->calls[i] = g_calls[i];
  }
  out->launches = g_launches.load();
  if (reset) {
    for (int i = 0; i < QOZ_PROF_STAGES; ++i) {
      g_ms[i] = 0.0;
      g_calls[i] = 0;
    }
    g_launches.store(0);
  }
  return QOZ_OK;
}

}  // extern "C"
