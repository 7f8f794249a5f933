// qrtebd_zgemm_noalloc: the tensor-core complex GEMM for callers that cannot
// allocate device memory.
//
// Some callers of this library cannot call cudaMalloc around a GEMM: code recorded
// into a CUDA graph under a capture mode that forbids allocation, latency-critical
// loops where an allocation (and the device-wide synchronisation of a later free)
// is not acceptable, and host frameworks that own all device memory through their
// own pool and do not hand out scratch. For them this entry point keeps its scratch
// - the split/embedded TF32 operands and the split-K partial sums - in one
// file-scope device array of fixed size, so a call allocates nothing. The caller
// still passes the inputs and the output.
//
// The array lives on every GPU that loads the library until the process exits.
// All calls share it and it keeps the previous call's contents; every element a
// call reads was written earlier in the same call, so nothing needs clearing, but
// calls that overlap on the GPU (different streams, or different host threads)
// race on it and must be serialised by the caller.
#include <mutex>

#include "tc_gemm.cuh"

namespace qrtebd {

namespace {

constexpr int kMaxDim = QRTEBD_NOALLOC_MAX_DIM;
constexpr size_t kLd = 2 * kMaxDim;                        // floats per operand row (2K, 128-B multiple)
constexpr size_t kA = (size_t)kMaxDim * kLd;               // floats per A' part (hi or lo)
constexpr size_t kB = (size_t)2 * kMaxDim * kLd;           // floats per B'^T part
constexpr size_t kP = (size_t)1 << 20;                     // split-K partial sums (floats)
constexpr size_t kFloats = 2 * kA + 2 * kB + kP;
static_assert(kFloats * sizeof(float) == (size_t)QRTEBD_NOALLOC_SCRATCH_BYTES,
              "scratch size must match the header");

__device__ __align__(256) float g_noalloc_scratch[kFloats];

std::mutex g_mu;
float* g_ptr[64] = {};

// Device address of the scratch array on the current device (set up once per device).
int scratch_address(float** out) {
  int dev = 0;
  QR_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) { set_last_message("zgemm_noalloc: device index out of range"); return QRTEBD_ERR_INVALID_ARG; }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_ptr[dev]) {
    void* p = nullptr;
    QR_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_ptr[dev] = static_cast<float*>(p);
  }
  *out = g_ptr[dev];
  return QRTEBD_OK;
}

}  // namespace
}  // namespace qrtebd

using namespace qrtebd;

extern "C" int qrtebd_zgemm_noalloc(int precision, int m, int n, int k, const void* A,
                                    long long sam, long long sak, int conj_a, const void* B,
                                    long long sbk, long long sbn, int conj_b, void* C,
                                    long long scm, long long scn, const double* alpha,
                                    const double* beta, void* stream) {
  if (precision != QRTEBD_C64_3XTF32 && precision != QRTEBD_C64_TF32) {
    set_last_message("zgemm_noalloc: only the tensor-core precisions C64_3XTF32 / C64_TF32");
    return QRTEBD_ERR_INVALID_ARG;
  }
  if (m < 0 || n < 0 || k < 0 || !A || !B || !C || !alpha || !beta) return QRTEBD_ERR_INVALID_ARG;
  if (m > kMaxDim || n > kMaxDim || k > kMaxDim) {
    set_last_message("zgemm_noalloc: m, n and k must not exceed QRTEBD_NOALLOC_MAX_DIM (512)");
    return QRTEBD_ERR_INVALID_ARG;
  }
  if (m == 0 || n == 0) return QRTEBD_OK;  // an empty C: nothing to write
  if (k == 0) {  // C = beta C: the CUDA-core kernel, which needs no scratch
    GemmArgs<float> g0{m, n, 0, static_cast<const float2*>(A), sam, sak, false,
                       static_cast<const float2*>(B), sbk, sbn, false, static_cast<float2*>(C), scm, scn,
                       make_float2((float)alpha[0], (float)alpha[1]), make_float2((float)beta[0], (float)beta[1])};
    ProfSuppress no_events;
    return gemm_simt<float>(g0, static_cast<cudaStream_t>(stream), nullptr, 0);
  }
  float* base = nullptr;
  QR_TRY(scratch_address(&base));
  // carve the fixed array: one A' slot (no caching across calls), B'^T, partial sums
  TcWorkspace w;
  w.a[0].hi = base;
  w.a[0].lo = base + kA;
  w.a[1] = w.a[0];
  w.b.hi = base + 2 * kA;
  w.b.lo = base + 2 * kA + kB;
  w.partial = base + 2 * kA + 2 * kB;
  w.a_cap = kA;
  w.b_cap = kB;
  w.p_cap = kP;
  GemmArgs<float> g{m, n, k, static_cast<const float2*>(A), sam, sak, conj_a != 0,
                    static_cast<const float2*>(B), sbk, sbn, conj_b != 0,
                    static_cast<float2*>(C), scm, scn,
                    make_float2((float)alpha[0], (float)alpha[1]),
                    make_float2((float)beta[0], (float)beta[1])};
  ProfSuppress no_events;  // profiling would create CUDA events
  return tc_gemm(g, precision == QRTEBD_C64_3XTF32, w, static_cast<cudaStream_t>(stream));
}
