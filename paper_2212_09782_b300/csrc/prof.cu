// Launch accounting and optional CUDA-event timing of kernel families.
//
// Every kernel launch of the library calls note_launch(); ProfScope brackets the
// launches of one family with CUDA events recorded on the launching stream when
// profiling is enabled (qrtebd_profile_enable), so a caller can read the average
// device duration of, e.g., the tensor-core GEMM from inside a timed region.
#include <atomic>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace qrtebd {

namespace {
std::atomic<long long> g_launches{0};
std::mutex g_mu;
bool g_enabled = false;
struct Rec { int fam; cudaEvent_t a, b; double flops; double bytes; };
std::vector<Rec> g_recs;       // recorded this window
std::vector<cudaEvent_t> g_free;  // event pool
cudaEvent_t take_event() {
  if (!g_free.empty()) { cudaEvent_t e = g_free.back(); g_free.pop_back(); return e; }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}
}  // namespace

thread_local int t_suppress = 0;

void note_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

ProfSuppress::ProfSuppress() { ++t_suppress; }
ProfSuppress::~ProfSuppress() { --t_suppress; }

ProfScope::ProfScope(int fam, cudaStream_t st, double flops, double bytes)
    : fam_(fam), st_(st), flops_(flops), bytes_(bytes) {
  if (t_suppress) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_enabled) return;
  a_ = take_event();
  b_ = take_event();
  if (a_ && b_) cudaEventRecord(static_cast<cudaEvent_t>(a_), st_);
}

ProfScope::~ProfScope() {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!a_ || !b_) return;
  cudaEventRecord(static_cast<cudaEvent_t>(b_), st_);
  g_recs.push_back(Rec{fam_, static_cast<cudaEvent_t>(a_), static_cast<cudaEvent_t>(b_), flops_, bytes_});
}

}  // namespace qrtebd

using namespace qrtebd;

extern "C" {

long long qrtebd_launch_count(void) { return g_launches.load(); }

int qrtebd_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& r : g_recs) { g_free.push_back(r.a); g_free.push_back(r.b); }
  g_recs.clear();
  g_enabled = (on != 0);
  return QRTEBD_OK;
}

int qrtebd_profile_read(int family, double* total_ms, long long* launches, double* flops,
                        double* bytes) {
  if (family < 0 || family >= PROF_NFAM) return QRTEBD_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_mu);
  double t = 0, f = 0, by = 0;
  long long n = 0;
  for (auto& r : g_recs) {
    if (r.fam != family) continue;
    QR_CUDA_TRY(cudaEventSynchronize(r.b));
    float ms = 0;
    QR_CUDA_TRY(cudaEventElapsedTime(&ms, r.a, r.b));
    t += ms; f += r.flops; by += r.bytes; ++n;
  }
  if (total_ms) *total_ms = t;
  if (launches) *launches = n;
  if (flops) *flops = f;
  if (bytes) *bytes = by;
  return QRTEBD_OK;
}

}  // extern "C"
