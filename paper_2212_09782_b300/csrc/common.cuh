// Shared device/host helpers for libqrtebd (sm_103a).
//
// Complex numbers are stored interleaved (re, im) as float2 (complex64) or
// double2 (complex128); every matrix is row-major with an explicit leading
// dimension counted in complex elements.
#pragma once

#include <cuda_runtime.h>
#include <utility>
#include <stdint.h>
#include <stdio.h>

#include <algorithm>
#include <cmath>
#include <type_traits>

#include "../../include/qrtebd.h"

namespace qrtebd {

// ---------------------------------------------------------------- complex
template <typename T> struct cplx;
template <> struct cplx<float> { using type = float2; };
template <> struct cplx<double> { using type = double2; };
template <typename T> using cx = typename cplx<T>::type;

template <typename T> __host__ __device__ __forceinline__ cx<T> mk(T r, T i) {
  cx<T> z; z.x = r; z.y = i; return z;
}
template <typename T> __host__ __device__ __forceinline__ cx<T> cadd(cx<T> a, cx<T> b) {
  return mk<T>(a.x + b.x, a.y + b.y);
}
template <typename T> __host__ __device__ __forceinline__ cx<T> csub(cx<T> a, cx<T> b) {
  return mk<T>(a.x - b.x, a.y - b.y);
}
template <typename T> __host__ __device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) {
  return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T> __host__ __device__ __forceinline__ cx<T> cconj(cx<T> a) {
  return mk<T>(a.x, -a.y);
}
// conj(a) * b
template <typename T> __host__ __device__ __forceinline__ cx<T> cmulc(cx<T> a, cx<T> b) {
  return mk<T>(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
// acc += a * b
template <typename T> __device__ __forceinline__ void cfma(cx<T>& acc, cx<T> a, cx<T> b) {
  acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
}
template <typename T> __host__ __device__ __forceinline__ T cabs2(cx<T> a) {
  return a.x * a.x + a.y * a.y;
}

// ---------------------------------------------------------------- errors
// Device-side error word: kernels that give up a bounded wait set a bit here
// and return; the host maps it to QRTEBD_ERR_TIMEOUT at the next sync point.
enum : unsigned { DEVERR_TIMEOUT = 1u, DEVERR_NUMERIC = 2u, DEVERR_BOUNDS = 4u };

// How many bond updates the enqueuing host thread runs at the same time (1: one alone),
// for the lifetime of a ConcurrencyScope (set by the layer executor and by the
// charge-sector update around their enqueues; defined in qr.cu). Launch shapes chosen to
// fill an otherwise idle GPU take a share of it instead: the QR's cooperative narrow
// updates (whose CTAs hold their SMs at the grid barriers until the grid's last CTA runs)
// and the tensor-core GEMM's K-splits (each split adds a partial-sum pass).
class ConcurrencyScope {
 public:
  explicit ConcurrencyScope(int n);
  ~ConcurrencyScope();
  ConcurrencyScope(const ConcurrencyScope&) = delete;
  ConcurrencyScope& operator=(const ConcurrencyScope&) = delete;

 private:
  int prev_;
};
int concurrency();

// Iteration limit for every spin on an mbarrier or a flag (~1 s on B300).
constexpr long long kSpinLimit = 1ll << 24;

// Poll limit of the grid-wide barriers (waits on a counter other CTAs advance, with no
// asynchronous copy in flight): each translation unit keeps a device copy, which
// qrtebd_set_spin_limit rewrites on the current device. The mbarrier waits of the TMA and
// cluster pipelines keep the compile-time kSpinLimit, since their expiry path drains
// copies still in flight and a tiny limit would cut that short.
static __device__ long long g_barrier_spin = kSpinLimit;
// Host side: records one translation unit's copy (its host shadow symbol); defined in capi.cu.
int register_barrier_spin(const void* host_symbol);
namespace {
[[maybe_unused]] const int g_barrier_spin_registered = register_barrier_spin(&g_barrier_spin);
}

#define QR_CUDA_TRY(expr)                                                           \
  do {                                                                              \
    cudaError_t e_ = (expr);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      qrtebd::set_last_error(e_, #expr, __FILE__, __LINE__);                        \
      return QRTEBD_ERR_CUDA;                                                       \
    }                                                                               \
  } while (0)

#define QR_TRY(expr)                                                                \
  do {                                                                              \
    int s_ = (expr);                                                                \
    if (s_ != QRTEBD_OK) return s_;                                                 \
  } while (0)

void set_last_error(cudaError_t e, const char* what, const char* file, int line);
void set_last_message(const char* msg);

// Address of the library's device error word on the current device (kernels
// atomicOr DEVERR_* bits into it; qrtebd_stream_check reads and clears it).
unsigned* device_error_word();

// Kernel-launch accounting (every launch site calls it) and event timing of
// kernel families (see prof.cu and qrtebd_profile_enable).
void note_launch(int n = 1);
enum ProfFamily { PROF_TC_GEMM = 0, PROF_QR_PANEL = 1, PROF_SIMT_GEMM = 2, PROF_PREP = 3,
                  PROF_GATE = 4, PROF_BOND_GEMM = 5, PROF_NFAM = 6 };
// While a ProfSuppress is alive on this thread, ProfScope records nothing (used by
// entry points that must not create CUDA objects).
struct ProfSuppress {
  ProfSuppress();
  ~ProfSuppress();
};
class ProfScope {
 public:
  ProfScope(int fam, cudaStream_t st, double flops = 0, double bytes = 0);
  ~ProfScope();
 private:
  int fam_; cudaStream_t st_; double flops_, bytes_;
  void* a_ = nullptr; void* b_ = nullptr;
};

// Programmatic dependent launch. A kernel started by launch_pdl() may be scheduled
// while the previous kernel on its stream is still draining (its launch latency and
// prologue overlap that kernel's tail); it calls pdl_wait() before its first access to
// global memory, which returns once every earlier kernel on the stream has completed
// and its writes are visible. pdl_launch_dependents() lets the next such kernel be
// scheduled as soon as every CTA of this one has started. Launched without the
// attribute, both are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// Grid-wide barrier of a cooperative launch (every CTA resident): a generation counter in
// bar[1] and an arrival count in bar[0] (both zero before the launch). The wait is bounded
// (kSpinLimit polls): on expiry DEVERR_TIMEOUT is set and false returned, and the caller
// must leave the kernel.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned nblocks, unsigned* err) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned* gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();
    if (atomicAdd(bar, 1u) == nblocks - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long long i = 0;
      const long long lim = g_barrier_spin;
      while (*gen == g) {
        if (++i > lim) { ok = 0; atomicOr(err, DEVERR_TIMEOUT); break; }
        __nanosleep(64);
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// complex128 storage (FP64 arithmetic, or FP64 emulated on the tensor cores)
inline bool prec_is_c128(int p) { return p == QRTEBD_C128 || p == QRTEBD_C128_OZ; }
inline bool prec_valid(int p) { return p >= QRTEBD_C128 && p <= QRTEBD_C128_OZ; }

__host__ __device__ __forceinline__ long long ceil_div(long long a, long long b) {
  return (a + b - 1) / b;
}
__host__ __device__ __forceinline__ size_t align_up(size_t x, size_t a) {
  return (x + a - 1) / a * a;
}

// Bump allocator over a caller-provided workspace; used to carve scratch.
struct Arena {
  char* base = nullptr;
  size_t cap = 0;
  size_t off = 0;
  bool measuring = false;  // size-query mode: hands out nullptr, only counts
  template <typename P> P* take(size_t count) {
    size_t bytes = align_up(count * sizeof(P), 256);
    size_t o = off;
    off += bytes;
    if (measuring) return nullptr;
    if (off > cap) return nullptr;
    return reinterpret_cast<P*>(base + o);
  }
  bool overflow() const { return !measuring && off > cap; }
};

}  // namespace qrtebd
