// Complex64 GEMM on tcgen05 tensor cores; see tc_gemm.cuh.
//
// Kernel: one 128 x 256 real output tile per CTA (one CTA per SM: ~197 KB of
// shared memory), 320 threads in three roles:
//   warp 0      TMA producer: 128B-swizzled K-major tiles of A' (128 x 32 fp32) and
//               B'^T (256 x 32 fp32) per stage, hi and lo parts, into a ring of
//               stages guarded by full/empty mbarriers;
//   warp 1      TMEM allocation (512 columns) and the single MMA-issuing thread:
//               per stage 4 K-steps of tcgen05.mma.kind::tf32 M=128 N=256 K=8
//               (x3 for hi*hi, hi*lo, lo*hi), tcgen05.commit frees the stage;
//   warps 2-9   epilogue: every 2 (3xTF32) or 4 stages the accumulator (two TMEM buffers,
//               ping-pong) is added into FP32 registers, one row and 128 columns
//               per thread; at the end alpha/beta and complex stores.
// The promotion matters: the tensor core's own accumulation loses low-order bits
// at every step, so accumulating all of K in TMEM gives an error growing like K
// rather than sqrt(K); chunked promotion restores FP32-like accuracy.
// Every mbarrier wait is bounded (kSpinLimit); on expiry the kernel sets
// DEVERR_TIMEOUT in the error word, drains what it issued and returns.
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include <atomic>
#include <map>
#include <mutex>

#include "tc_gemm.cuh"

namespace qrtebd {

namespace {

constexpr int BM = 128, BK = 32;               // BK in fp32 elements = one 128 B swizzle row
constexpr int A_TILE = BM * BK * 4;            // 16 KB
constexpr int NEPI = 8;                         // epilogue warps
constexpr int NTHREADS = 64 + 32 * NEPI;        // producer, MMA, epilogue
constexpr int CHUNK = 4;                        // stages per FP32 promotion (1xTF32; the split
                                                // heuristics' unit of K)
// 3xTF32 promotes every 2 stages: a chunk then builds 24 tensor-core accumulations on each
// other instead of 48. The accumulation in TMEM truncates, so its error is a bias that
// shrinks norms; at 48 it set the complex64 CBE update's eps error (8e-6 relative on an
// eta = 351 bond, against 1.3e-6 with FP32 CUDA-core products)
template <bool THREE> constexpr int promo_chunk() { return THREE ? 2 : CHUNK; }

// BN: real output columns per tile (256, or 128 for narrow or few-tile products); the
// stage ring fills ~192 KB of shared memory either way
template <bool THREE, int BN> struct Cfg {
  static_assert(BN == 128 || BN == 256, "tile width");
  static constexpr int B_TILE = BN * BK * 4;            // 32 or 16 KB
  static constexpr int TMEM_COLS = 2 * BN;              // two accumulators
  static constexpr int STAGE_BYTES = THREE ? 2 * (A_TILE + B_TILE) : (A_TILE + B_TILE);
  static constexpr int STAGES = (192 * 1024) / STAGE_BYTES;
  static constexpr int SMEM = STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;
  // instruction descriptor: D fp32, A/B tf32, both K-major, M = BM, N = BN
  static constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) |
                                    ((uint32_t)(BM >> 4) << 24);
};

struct Epi {
  float2* C; long long scm, scn;
  float2 alpha, beta;
  int M, Nc;  // rows, complex columns
};

__device__ __forceinline__ uint32_t s_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s_u32(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s_u32(b)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(s_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity) {
  for (long long i = 0; i < kSpinLimit; ++i)
    if (mbar_try(b, parity)) return true;
  return false;
}
__device__ __forceinline__ void tma_load(void* dst, const CUtensorMap* tm, uint64_t* bar, int x,
                                         int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(s_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(s_u32(bar)), "r"(x), "r"(y)
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
// the same with FP16 operands (both A and B f16), FP32 accumulation
__device__ __forceinline__ void tc_mma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                           uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          s_u32(bar))
      : "memory");
}
// K-major operand tile, 128-byte swizzle: rows of 128 B, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;                // leading byte offset (unused for SW128 K-major)
  d |= (uint64_t)(1024 >> 4) << 32;      // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                // descriptor version (tcgen05)
  d |= (uint64_t)2 << 61;                // 128-byte swizzle
  return d;
}

#define TMEM_LD32(taddr, r)                                                                  \
  asm volatile(                                                                              \
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13," \
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"     \
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),  \
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),          \
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),       \
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),       \
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),       \
        "=r"(r[31])                                                                          \
      : "r"(taddr))

#define TMEM_ST32(taddr, r)                                                                  \
  asm volatile(                                                                              \
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"  \
      "%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};"     \
      ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), \
        "r"(r[7]), "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]),     \
        "r"(r[14]), "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]),  \
        "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]),  \
        "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])                                       \
      : "memory")

#define TMEM_LD16(taddr, r)                                                                  \
  asm volatile(                                                                              \
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13," \
      "%14,%15}, [%16];"                                                                     \
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),  \
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),          \
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])                                                \
      : "r"(taddr))

__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(s_u32(b)) : "memory");
}

// Kernel. Roles: warp 0 TMA producer, warp 1 TMEM allocator + MMA issuer, warps
// 2..9 epilogue. The K loop is cut into chunks of promo_chunk() stages; each chunk
// accumulates into one of two TMEM buffers (columns [0,256) and [256,512)) and the
// epilogue warps add every finished chunk into FP32 registers (each thread one row,
// 128 columns), so at most 4*2*3 (3xTF32) or 4*4 tensor-core accumulations build on each other
// before a correctly rounded FP32 add. grid.z splits K (partial != nullptr: raw
// partial sums are written for a separate reduction).
template <bool THREE, int BN>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap tA_hi, const __grid_constant__ CUtensorMap tA_lo,
              const __grid_constant__ CUtensorMap tB_hi, const __grid_constant__ CUtensorMap tB_lo,
              Epi epi, int Kp, int kt_per_split, float* partial, int m_off, unsigned* err,
              int ktri) {
  // m_off: first row of this launch's tiles in A; the epilogue's rows (and epi) are
  // relative to it. ktri: the product's operands are triangular, so a tile's K loop ends
  // early: 1 = A' lower triangular (real K below 2 (last row of the tile + 1)), 2 = B'^T
  // upper triangular along K (real K below the tile's last real column + 1); 0 = full K.
  // The K-tiles skipped hold only zeros of the triangular operand.
  using C = Cfg<THREE, BN>;
  constexpr int B_TILE = C::B_TILE, TMEM_COLS = C::TMEM_COLS;
  static_assert(BM * (BN + 4) * 4 <= C::STAGES * C::STAGE_BYTES, "staged epilogue tile");
  constexpr uint32_t kIdesc = C::IDESC;
  constexpr int HW = BN / 2;  // columns per epilogue thread
  pdl_launch_dependents();
  pdl_wait();
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = smem_raw + ((1024 - (s_u32(smem_raw) & 1023)) & 1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + C::STAGES * C::STAGE_BYTES);
  uint64_t* empty = full + C::STAGES;
  uint64_t* accf = empty + C::STAGES;  // [2] chunk accumulated
  uint64_t* acce = accf + 2;           // [2] chunk drained
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acce + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n0 = blockIdx.x * BN, m0 = blockIdx.y * BM;
  int kreal = Kp;
  if (ktri == 1) kreal = min(Kp, 2 * (m_off + m0 + BM));
  else if (ktri == 2) kreal = min(Kp, n0 + BN);
  const int nk_all = (kreal + BK - 1) / BK;
  const int kt0 = blockIdx.z * kt_per_split;
  const int kt1 = min(nk_all, kt0 + kt_per_split);
  const int nk = max(0, kt1 - kt0);
  constexpr int KCH = promo_chunk<THREE>();
  const int nchunks = (nk + KCH - 1) / KCH;

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(&accf[b], 1); mbar_init(&acce[b], NEPI); }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     s_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  auto stage_a_hi = [&](int s) { return smem + s * C::STAGE_BYTES; };
  auto stage_b_hi = [&](int s) { return smem + s * C::STAGE_BYTES + A_TILE; };
  auto stage_a_lo = [&](int s) { return smem + s * C::STAGE_BYTES + A_TILE + B_TILE; };
  auto stage_b_lo = [&](int s) { return smem + s * C::STAGE_BYTES + 2 * A_TILE + B_TILE; };

  if (warp == 0) {
    if (lane == 0) {
      bool ok = true;
      int issued = 0;
      for (int i = 0; i < nk && ok; ++i) {
        const int s = i % C::STAGES;
        const uint32_t ph = (uint32_t)((i / C::STAGES) & 1);
        if (!mbar_wait(&empty[s], ph ^ 1u)) { ok = false; break; }
        const int kx = (kt0 + i) * BK;
        mbar_expect_tx(&full[s], C::STAGE_BYTES);
        tma_load(stage_a_hi(s), &tA_hi, &full[s], kx, m0 + m_off);
        tma_load(stage_b_hi(s), &tB_hi, &full[s], kx, n0);
        if (THREE) {
          tma_load(stage_a_lo(s), &tA_lo, &full[s], kx, m0 + m_off);
          tma_load(stage_b_lo(s), &tB_lo, &full[s], kx, n0);
        }
        ++issued;
      }
      if (!ok) atomicOr(err, DEVERR_TIMEOUT);
      // drain: every issued stage must have landed before shared memory goes away
      for (int i = (issued > C::STAGES ? issued - C::STAGES : 0); i < issued; ++i) {
        if (!mbar_wait(&full[i % C::STAGES], (uint32_t)((i / C::STAGES) & 1))) {
          atomicOr(err, DEVERR_TIMEOUT);
          break;
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      bool ok = true;
      for (int c = 0; c < nchunks && ok; ++c) {
        const int b = c & 1;
        if (c >= 2 && !mbar_wait(&acce[b], (uint32_t)(((c >> 1) - 1) & 1))) { ok = false; break; }
        tc_fence_after();
        const uint32_t acc_t = tmem + (uint32_t)(b * BN);
        const int i1 = min(nk, (c + 1) * KCH);
        for (int i = c * KCH; i < i1; ++i) {
          const int s = i % C::STAGES;
          if (!mbar_wait(&full[s], (uint32_t)((i / C::STAGES) & 1))) { ok = false; break; }
          tc_fence_after();
          const uint32_t a_hi = s_u32(stage_a_hi(s)), b_hi = s_u32(stage_b_hi(s));
          const uint32_t a_lo = s_u32(stage_a_lo(s)), b_lo = s_u32(stage_b_lo(s));
#pragma unroll
          for (int k = 0; k < BK / 8; ++k) {
            const uint32_t off = k * 32;  // 8 tf32 = 32 bytes along K inside the swizzle row
            const uint32_t acc = (i > c * KCH || k > 0) ? 1u : 0u;
            if (THREE) {
              tc_mma(acc_t, desc_sw128(a_lo + off), desc_sw128(b_hi + off), kIdesc, acc);
              tc_mma(acc_t, desc_sw128(a_hi + off), desc_sw128(b_lo + off), kIdesc, 1u);
              tc_mma(acc_t, desc_sw128(a_hi + off), desc_sw128(b_hi + off), kIdesc, 1u);
            } else {
              tc_mma(acc_t, desc_sw128(a_hi + off), desc_sw128(b_hi + off), kIdesc, acc);
            }
          }
          tc_commit(&empty[s]);
        }
        tc_commit(&accf[b]);  // fires once this chunk's MMAs have completed
      }
      if (!ok) atomicOr(err, DEVERR_TIMEOUT);
    }
  } else {
    // epilogue warps 2..9: TMEM lane quarter q, column half h
    const int q = warp & 3;
    const int h = (warp - 2) >> 2;
    const int row = m0 + q * 32 + lane;
    float sum[HW];
#pragma unroll
    for (int j = 0; j < HW; ++j) sum[j] = 0.f;
    bool ok = true;
    for (int c = 0; c < nchunks; ++c) {
      const int b = c & 1;
      if (!mbar_wait(&accf[b], (uint32_t)((c >> 1) & 1))) { ok = false; break; }
      tc_fence_after();
#pragma unroll
      for (int blk = 0; blk < HW / 32; ++blk) {
        uint32_t r[32];
        const uint32_t taddr =
            tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * BN + h * HW + blk * 32);
        TMEM_LD32(taddr, r);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int j = 0; j < 32; ++j) sum[blk * 32 + j] += __uint_as_float(r[j]);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acce[b]);
    }
    if (!ok && lane == 0) atomicOr(err, DEVERR_TIMEOUT);
    if (partial || epi.scn == 1) {
      // Rows of the output are contiguous: stage the tile in the idle pipeline buffers
      // (every MMA has completed) so that each warp then reads and writes whole row
      // segments - coalesced - instead of one row per thread.
      constexpr int LDT = BN + 4;  // floats per staged row; conflict-free float4 stores
      float* tile = reinterpret_cast<float*>(smem);
      if (ok) {
        float* trow = tile + (q * 32 + lane) * LDT + h * HW;
#pragma unroll
        for (int j = 0; j < HW; j += 4)
          *reinterpret_cast<float4*>(trow + j) = make_float4(sum[j], sum[j + 1], sum[j + 2], sum[j + 3]);
      }
      asm volatile("bar.sync 1, %0;" ::"n"(32 * NEPI) : "memory");
      if (ok) {
        const bool use_beta = (epi.beta.x != 0.f || epi.beta.y != 0.f);
        for (int r = warp - 2; r < BM; r += NEPI) {
          const int grow = m0 + r;
          if (grow >= epi.M) break;
          const float* tr = tile + r * LDT;
          if (partial) {
            float* prow = partial + ((long long)blockIdx.z * epi.M + grow) * (2LL * epi.Nc);
            for (int j = lane; j < BN; j += 32)
              if (n0 + j < 2 * epi.Nc) prow[n0 + j] = tr[j];
          } else {
            float2* crow = epi.C + (long long)grow * epi.scm;
            for (int c = lane; c < BN / 2; c += 32) {
              const int n = n0 / 2 + c;
              if (n < epi.Nc) {
                const float2 a = *reinterpret_cast<const float2*>(tr + 2 * c);
                float2 v;
                v.x = epi.alpha.x * a.x - epi.alpha.y * a.y;
                v.y = epi.alpha.x * a.y + epi.alpha.y * a.x;
                if (use_beta) {
                  const float2 cv = crow[n];
                  v.x += epi.beta.x * cv.x - epi.beta.y * cv.y;
                  v.y += epi.beta.x * cv.y + epi.beta.y * cv.x;
                }
                crow[n] = v;
              }
            }
          }
        }
      }
    } else if (ok && row < epi.M) {
      // general strides (a transposed output is coalesced across the warp's rows)
      const int col0 = n0 + h * HW;  // first real column of this thread's half
      const bool use_beta = (epi.beta.x != 0.f || epi.beta.y != 0.f);
      float2* crow = epi.C + (long long)row * epi.scm;
#pragma unroll
      for (int j = 0; j < HW / 2; ++j) {
        const int n = (col0 >> 1) + j;
        if (n < epi.Nc) {
          const float ar = sum[2 * j], ai = sum[2 * j + 1];
          float2 v;
          v.x = epi.alpha.x * ar - epi.alpha.y * ai;
          v.y = epi.alpha.x * ai + epi.alpha.y * ar;
          float2* p = crow + (long long)n * epi.scn;
          if (use_beta) {
            const float2 cv = *p;
            v.x += epi.beta.x * cv.x - epi.beta.y * cv.y;
            v.y += epi.beta.x * cv.y + epi.beta.y * cv.x;
          }
          *p = v;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    // every chunk commit has fired (the epilogue waited on them) unless a wait
    // expired; wait once more (bounded) so no MMA still writes the columns being freed
    if (nchunks > 0) {
      const int c = nchunks - 1;
      if (!mbar_wait(&accf[c & 1], (uint32_t)((c >> 1) & 1)) && lane == 0)
        atomicOr(err, DEVERR_TIMEOUT);
    }
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
  }
}

// C = alpha * sum_z partial[z] + beta * C (partials: split x M x 2N floats)
__global__ void k_splitk_sum(const float* partial, int splits, Epi epi) {
  pdl_launch_dependents();
  pdl_wait();
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long MN = (long long)epi.M * epi.Nc;
  if (idx >= MN) return;
  const int m = (int)(idx / epi.Nc), n = (int)(idx % epi.Nc);
  float ar = 0.f, ai = 0.f;
  for (int z = 0; z < splits; ++z) {
    const float* p = partial + ((long long)z * epi.M + m) * (2LL * epi.Nc) + 2 * n;
    ar += p[0]; ai += p[1];
  }
  float2 v;
  v.x = epi.alpha.x * ar - epi.alpha.y * ai;
  v.y = epi.alpha.x * ai + epi.alpha.y * ar;
  float2* c = epi.C + (long long)m * epi.scm + (long long)n * epi.scn;
  if (epi.beta.x != 0.f || epi.beta.y != 0.f) {
    const float2 cv = *c;
    v.x += epi.beta.x * cv.x - epi.beta.y * cv.y;
    v.y += epi.beta.x * cv.y + epi.beta.y * cv.x;
  }
  *c = v;
}

// ------------------------------------------------------------------ prep
__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// A'[m][2k..2k+1] = (Re, Im) opA(m, k), split hi/lo; one 32 x 32 tile (bx, by)
__device__ __forceinline__ void prep_a_tile(const float2* __restrict__ A, long long sam, long long sak,
                                            int conj, int M, int K, float* __restrict__ hi,
                                            float* __restrict__ lo, int ld, int three, int bx, int by,
                                            float2 (*t)[33]) {
  const int m0 = by * 32, k0 = bx * 32;
  const bool kc = (sak == 1);
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    int mm = kc ? r : threadIdx.x, kk = kc ? threadIdx.x : r;
    int m = m0 + mm, k = k0 + kk;
    float2 v = make_float2(0.f, 0.f);
    if (m < M && k < K) v = A[m * sam + k * sak];
    if (conj) v.y = -v.y;
    t[mm][kk] = v;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    int m = m0 + r, k = k0 + threadIdx.x;
    if (m < M && k < K) {
      float2 v = t[r][threadIdx.x];
      float2 h = make_float2(tf32_rna(v.x), tf32_rna(v.y));
      long long o = (long long)m * ld + 2 * k;
      *reinterpret_cast<float2*>(hi + o) = h;
      if (three) *reinterpret_cast<float2*>(lo + o) = make_float2(v.x - h.x, v.y - h.y);
    }
  }
}

// B'^T rows 2n: (Re b, -Im b), 2n+1: (Im b, Re b) at columns 2k, 2k+1; b = opB(k, n)
__device__ __forceinline__ void prep_b_tile(const float2* __restrict__ B, long long sbk, long long sbn,
                                            int conj, int K, int N, float* __restrict__ hi,
                                            float* __restrict__ lo, int ld, int three, int bx, int by,
                                            float2 (*t)[33]) {  // t: [n][k]
  const int n0 = by * 32, k0 = bx * 32;
  const bool kc = (sbk == 1);
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    int nn = kc ? r : threadIdx.x, kk = kc ? threadIdx.x : r;
    int n = n0 + nn, k = k0 + kk;
    float2 v = make_float2(0.f, 0.f);
    if (n < N && k < K) v = B[k * sbk + n * sbn];
    if (conj) v.y = -v.y;
    t[nn][kk] = v;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    int n = n0 + r, k = k0 + threadIdx.x;
    if (n < N && k < K) {
      float2 b = t[r][threadIdx.x];
      float br = tf32_rna(b.x), bi = tf32_rna(b.y);
      long long o0 = (long long)(2 * n) * ld + 2 * k, o1 = o0 + ld;
      *reinterpret_cast<float2*>(hi + o0) = make_float2(br, -bi);
      *reinterpret_cast<float2*>(hi + o1) = make_float2(bi, br);
      if (three) {
        float lr = b.x - br, li = b.y - bi;
        *reinterpret_cast<float2*>(lo + o0) = make_float2(lr, -li);
        *reinterpret_cast<float2*>(lo + o1) = make_float2(li, lr);
      }
    }
  }
}

struct PrepJob {
  const float2* src; long long s0, s1; int conj, rows, K;
  float* hi; float* lo; int ld;
  int gx, gy;  // tiles along K and along rows
  int vec;     // 1: the operand is contiguous along K with 16-byte aligned pairs (vector form)
};

// Vector form for an operand contiguous along K (A: s1 = 1, rows m at stride s0; B: s0 = 1,
// columns n at stride s1): no transpose, so each thread converts two complex values at a
// time with one 16-byte load and 16-byte stores (the tile form stages a 32 x 32 tile in
// shared memory for every layout). The values written are the tile form's, bit for bit.
// Units (row, pair of K) are spread over every block of the operand's grid slice.
__device__ __forceinline__ void prep_vec(const PrepJob& j, bool embed, int three) {
  const unsigned kp = (unsigned)(j.K + 1) >> 1;
  const unsigned units = (unsigned)j.rows * kp;  // < 2^31 (host-checked)
  const unsigned nthr = gridDim.x * gridDim.y * blockDim.x * blockDim.y;
  const long long rs = embed ? j.s1 : j.s0;
  for (unsigned u = (blockIdx.y * gridDim.x + blockIdx.x) * (blockDim.x * blockDim.y) +
                    threadIdx.y * blockDim.x + threadIdx.x;
       u < units; u += nthr) {
    const unsigned r = u / kp;
    const int k = 2 * (int)(u - r * kp);
    const float2* p = j.src + (long long)r * rs + k;
    const bool two = k + 1 < j.K;
    float4 v;
    if (two) v = *reinterpret_cast<const float4*>(p);
    else { const float2 x = *p; v = make_float4(x.x, x.y, 0.f, 0.f); }
    if (j.conj) { v.y = -v.y; v.w = -v.w; }
    const float4 h = make_float4(tf32_rna(v.x), tf32_rna(v.y), tf32_rna(v.z), tf32_rna(v.w));
    const float4 l = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
    if (!embed) {
      const long long o = (long long)r * j.ld + 2 * k;
      if (two) {
        *reinterpret_cast<float4*>(j.hi + o) = h;
        if (three) *reinterpret_cast<float4*>(j.lo + o) = l;
      } else {
        *reinterpret_cast<float2*>(j.hi + o) = make_float2(h.x, h.y);
        if (three) *reinterpret_cast<float2*>(j.lo + o) = make_float2(l.x, l.y);
      }
    } else {
      // B'^T rows 2n: (Re b, -Im b), 2n+1: (Im b, Re b)
      const long long o0 = (long long)(2 * r) * j.ld + 2 * k, o1 = o0 + j.ld;
      if (two) {
        *reinterpret_cast<float4*>(j.hi + o0) = make_float4(h.x, -h.y, h.z, -h.w);
        *reinterpret_cast<float4*>(j.hi + o1) = make_float4(h.y, h.x, h.w, h.z);
        if (three) {
          *reinterpret_cast<float4*>(j.lo + o0) = make_float4(l.x, -l.y, l.z, -l.w);
          *reinterpret_cast<float4*>(j.lo + o1) = make_float4(l.y, l.x, l.w, l.z);
        }
      } else {
        *reinterpret_cast<float2*>(j.hi + o0) = make_float2(h.x, -h.y);
        *reinterpret_cast<float2*>(j.hi + o1) = make_float2(h.y, h.x);
        if (three) {
          *reinterpret_cast<float2*>(j.lo + o0) = make_float2(l.x, -l.y);
          *reinterpret_cast<float2*>(j.lo + o1) = make_float2(l.y, l.x);
        }
      }
    }
  }
}

// One launch prepares both operands: blockIdx.z = 0 the A' tiles, 1 the B' tiles
// (tiles beyond an operand's own grid return at once); an operand in the vector form
// spreads its units over the whole of its grid slice.
__global__ void k_prep(PrepJob a, PrepJob b, int three) {
  __shared__ float2 t[32][33];
  pdl_launch_dependents();
  pdl_wait();
  const PrepJob& j = blockIdx.z == 0 ? a : b;
  if (j.vec) { prep_vec(j, blockIdx.z == 1, three); return; }
  if ((int)blockIdx.x >= j.gx || (int)blockIdx.y >= j.gy) return;
  if (blockIdx.z == 0)
    prep_a_tile(j.src, j.s0, j.s1, j.conj, j.rows, j.K, j.hi, j.lo, j.ld, three, blockIdx.x, blockIdx.y, t);
  else
    prep_b_tile(j.src, j.s0, j.s1, j.conj, j.K, j.rows, j.hi, j.lo, j.ld, three, blockIdx.x, blockIdx.y, t);
}

// ------------------------------------------------------------------ fused operand preparation
// The same GEMM with the operand preparation done in the kernel. The eight epilogue warps
// also convert: one stage ahead they read the raw complex64 operands (16-byte global loads
// of two complex values), split every value into its TF32 part and remainder (hi = tf32(x),
// lo = x - hi), and store A' and the 2 x 2 embedded B'^T directly into the stage buffers in
// the 128-byte-swizzled K-major layout a tiled TMA load would produce (16-byte chunk c of
// tile row r at byte r * 128 + ((c ^ (r & 7)) << 4), tiles 1024-byte aligned). A proxy fence
// makes these generic stores visible to the tensor core's reads before each warp arrives on
// the stage's full barrier. Between stages they drain finished accumulator chunks as before.
// Layouts handled: opA contiguous along K (sak = 1) or along M (sam = 1), opB contiguous
// along K (sbk = 1) or along N (sbn = 1), with 16-byte aligned pairs (checked on the host).
struct RawOp {
  const float2* p; long long s0, s1;  // A: (m, k) at p[m s0 + k s1]; B: (k, n) at p[k s0 + n s1]
  int conj, kmajor, rows, K;          // kmajor: A s1 == 1, B s0 == 1; rows: M (A) or N (B)
};

__device__ __forceinline__ float4 ld_pair(const float2* p, bool two, bool one) {
  if (two) return *reinterpret_cast<const float4*>(p);
  if (one) { const float2 v = *p; return make_float4(v.x, v.y, 0.f, 0.f); }
  return make_float4(0.f, 0.f, 0.f, 0.f);
}
__device__ __forceinline__ float4 conj4(float4 v, int c) { if (c) { v.y = -v.y; v.w = -v.w; } return v; }
__device__ __forceinline__ void split_store(uint8_t* hi, uint8_t* lo, uint32_t off, float4 v, bool three) {
  const float4 h = make_float4(tf32_rna(v.x), tf32_rna(v.y), tf32_rna(v.z), tf32_rna(v.w));
  *reinterpret_cast<float4*>(hi + off) = h;
  if (three) *reinterpret_cast<float4*>(lo + off) = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
}
__device__ __forceinline__ uint32_t sw128(int r, int c) { return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4)); }

// Raw values of stage i (complex K from (kt0 + i) * 16) for converter thread ct: A as four
// 16-byte chunks (K-major: tile row idx / 8, pair idx % 8) or two 2 x 2 blocks (M-major:
// M pair idx % 64, K pair idx / 64), idx = ct + 256 u; B likewise with BN / 2 columns.
template <int BN>
__device__ __forceinline__ void fz_load(float4 (&xa)[4], float4 (&xb)[BN / 64], const RawOp& ra, const RawOp& rb,
                                        int kt0, int i, int ct, long long ma0, int nc0, int Kc) {
  constexpr int NB = BN / 64;
  const int kc0 = (kt0 + i) * (BK / 2);
  if (ra.kmajor) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int idx = ct + 256 * u, r = idx >> 3, c = idx & 7;
      const long long m = ma0 + r;
      const int k = kc0 + 2 * c;
      const bool in = m < ra.rows;
      xa[u] = ld_pair(ra.p + m * ra.s0 + k, in && k + 1 < Kc, in && k < Kc);
    }
  } else {
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int idx = ct + 256 * u, mp = idx & 63, kp = idx >> 6;
      const long long m = ma0 + 2 * mp;
      const int k = kc0 + 2 * kp;
      const bool two = m + 1 < ra.rows, one = m < ra.rows;
      xa[2 * u] = ld_pair(ra.p + (long long)k * ra.s1 + m, two && k < Kc, one && k < Kc);
      xa[2 * u + 1] = ld_pair(ra.p + (long long)(k + 1) * ra.s1 + m, two && k + 1 < Kc, one && k + 1 < Kc);
    }
  }
  if (rb.kmajor) {
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      const int idx = ct + 256 * u, nl = idx >> 3, c = idx & 7;
      const long long n = nc0 + nl;
      const int k = kc0 + 2 * c;
      const bool in = n < rb.rows;
      xb[u] = ld_pair(rb.p + n * rb.s1 + k, in && k + 1 < Kc, in && k < Kc);
    }
  } else {
#pragma unroll
    for (int u = 0; u < NB / 2; ++u) {
      const int idx = ct + 256 * u, np = idx % (BN / 4), kp = idx / (BN / 4);
      const long long n = nc0 + 2 * np;
      const int k = kc0 + 2 * kp;
      const bool two = n + 1 < rb.rows, one = n < rb.rows;
      xb[2 * u] = ld_pair(rb.p + (long long)k * rb.s0 + n, two && k < Kc, one && k < Kc);
      xb[2 * u + 1] = ld_pair(rb.p + (long long)(k + 1) * rb.s0 + n, two && k + 1 < Kc, one && k + 1 < Kc);
    }
  }
}

// B'^T rows 2 nl: (Re b, -Im b), 2 nl + 1: (Im b, Re b) for the two K values of chunk c
__device__ __forceinline__ void fz_emb(uint8_t* bhi, uint8_t* blo, int nl, int c, float4 v, int conj, bool three) {
  v = conj4(v, conj);
  split_store(bhi, blo, sw128(2 * nl, c), make_float4(v.x, -v.y, v.z, -v.w), three);
  split_store(bhi, blo, sw128(2 * nl + 1, c), make_float4(v.y, v.x, v.w, v.z), three);
}

template <bool THREE, int BN>
__device__ __forceinline__ void fz_store(const float4 (&xa)[4], const float4 (&xb)[BN / 64], const RawOp& ra,
                                         const RawOp& rb, uint8_t* ahi, uint8_t* alo, uint8_t* bhi, uint8_t* blo,
                                         int ct) {
  constexpr int NB = BN / 64;
  if (ra.kmajor) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int idx = ct + 256 * u, r = idx >> 3, c = idx & 7;
      split_store(ahi, alo, sw128(r, c), conj4(xa[u], ra.conj), THREE);
    }
  } else {
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int idx = ct + 256 * u, mp = idx & 63, kp = idx >> 6;
      const float4 p0 = xa[2 * u], p1 = xa[2 * u + 1];  // (k, m m+1), (k+1, m m+1)
      split_store(ahi, alo, sw128(2 * mp, kp), conj4(make_float4(p0.x, p0.y, p1.x, p1.y), ra.conj), THREE);
      split_store(ahi, alo, sw128(2 * mp + 1, kp), conj4(make_float4(p0.z, p0.w, p1.z, p1.w), ra.conj), THREE);
    }
  }
  if (rb.kmajor) {
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      const int idx = ct + 256 * u;
      fz_emb(bhi, blo, idx >> 3, idx & 7, xb[u], rb.conj, THREE);
    }
  } else {
#pragma unroll
    for (int u = 0; u < NB / 2; ++u) {
      const int idx = ct + 256 * u, np = idx % (BN / 4), kp = idx / (BN / 4);
      const float4 p0 = xb[2 * u], p1 = xb[2 * u + 1];  // (k, n n+1), (k+1, n n+1)
      fz_emb(bhi, blo, 2 * np, kp, make_float4(p0.x, p0.y, p1.x, p1.y), rb.conj, THREE);
      fz_emb(bhi, blo, 2 * np + 1, kp, make_float4(p0.z, p0.w, p1.z, p1.w), rb.conj, THREE);
    }
  }
}

// 128-column tiles only: with ten warps one SM sub-partition holds three of them, so a
// thread has at most 168 registers, which a 256-column tile's 128 FP32 sums plus a stage of
// raw operand values in flight would exceed (such products keep the separate preparation)
template <bool THREE, int BN>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_tc_gemm_fz(RawOp ra, RawOp rb, Epi epi, int kt_per_split, float* partial, int m_off, unsigned* err) {
  using C = Cfg<THREE, BN>;
  constexpr int B_TILE = C::B_TILE, TMEM_COLS = C::TMEM_COLS;
  static_assert(BM * (BN + 4) * 4 <= C::STAGES * C::STAGE_BYTES, "staged epilogue tile");
  static_assert(BN == 128, "in-kernel preparation: 128-column tiles");
  constexpr uint32_t kIdesc = C::IDESC;
  constexpr int HW = BN / 2;   // columns per epilogue thread
  constexpr int NB = BN / 64;  // B chunks (or 2 x 2 blocks / 2) per converter thread
  pdl_launch_dependents();
  pdl_wait();
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = smem_raw + ((1024 - (s_u32(smem_raw) & 1023)) & 1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + C::STAGES * C::STAGE_BYTES);
  uint64_t* empty = full + C::STAGES;
  uint64_t* accf = empty + C::STAGES;
  uint64_t* acce = accf + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acce + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n0 = blockIdx.x * BN, m0 = blockIdx.y * BM;
  const int Kc = ra.K;                       // complex K
  const int nk_all = (2 * Kc + BK - 1) / BK;  // stages of 16 complex K
  const int kt0 = blockIdx.z * kt_per_split;
  const int kt1 = min(nk_all, kt0 + kt_per_split);
  const int nk = max(0, kt1 - kt0);
  constexpr int KCH = promo_chunk<THREE>();
  const int nchunks = (nk + KCH - 1) / KCH;

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) { mbar_init(&full[s], NEPI); mbar_init(&empty[s], 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(&accf[b], 1); mbar_init(&acce[b], NEPI); }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     s_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  auto stage_a_hi = [&](int s) { return smem + s * C::STAGE_BYTES; };
  auto stage_b_hi = [&](int s) { return smem + s * C::STAGE_BYTES + A_TILE; };
  auto stage_a_lo = [&](int s) { return smem + s * C::STAGE_BYTES + A_TILE + B_TILE; };
  auto stage_b_lo = [&](int s) { return smem + s * C::STAGE_BYTES + 2 * A_TILE + B_TILE; };

  if (warp == 1) {
    if (lane == 0) {
      bool ok = true;
      for (int c = 0; c < nchunks && ok; ++c) {
        const int b = c & 1;
        if (c >= 2 && !mbar_wait(&acce[b], (uint32_t)(((c >> 1) - 1) & 1))) { ok = false; break; }
        tc_fence_after();
        const uint32_t acc_t = tmem + (uint32_t)(b * BN);
        const int i1 = min(nk, (c + 1) * KCH);
        for (int i = c * KCH; i < i1; ++i) {
          const int s = i % C::STAGES;
          if (!mbar_wait(&full[s], (uint32_t)((i / C::STAGES) & 1))) { ok = false; break; }
          tc_fence_after();
          const uint32_t a_hi = s_u32(stage_a_hi(s)), b_hi = s_u32(stage_b_hi(s));
          const uint32_t a_lo = s_u32(stage_a_lo(s)), b_lo = s_u32(stage_b_lo(s));
#pragma unroll
          for (int k = 0; k < BK / 8; ++k) {
            const uint32_t off = k * 32;
            const uint32_t acc = (i > c * KCH || k > 0) ? 1u : 0u;
            if (THREE) {
              tc_mma(acc_t, desc_sw128(a_lo + off), desc_sw128(b_hi + off), kIdesc, acc);
              tc_mma(acc_t, desc_sw128(a_hi + off), desc_sw128(b_lo + off), kIdesc, 1u);
              tc_mma(acc_t, desc_sw128(a_hi + off), desc_sw128(b_hi + off), kIdesc, 1u);
            } else {
              tc_mma(acc_t, desc_sw128(a_hi + off), desc_sw128(b_hi + off), kIdesc, acc);
            }
          }
          tc_commit(&empty[s]);
        }
        tc_commit(&accf[b]);
      }
      if (!ok) atomicOr(err, DEVERR_TIMEOUT);
    }
  } else if (warp >= 2) {
    // converter + epilogue warps 2..9: TMEM lane quarter q, column half h
    const int q = warp & 3;
    const int h = (warp - 2) >> 2;
    const int ct = threadIdx.x - 64;  // 0 .. 255
    const int row = m0 + q * 32 + lane;
    const long long ma0 = (long long)m_off + m0;  // first row of opA in this tile
    const int nc0 = n0 / 2;                        // first complex column of opB in this tile
    float sum[HW];
#pragma unroll
    for (int j = 0; j < HW; ++j) sum[j] = 0.f;
    float4 xa[4], xb[NB];
    // raw values of stage i and their conversion into stage slot s (fz_load / fz_store)
    bool ok = true;
    int drained = 0;  // chunks added into the registers so far
    auto drain = [&](int c) {
      const int b = c & 1;
      if (!mbar_wait(&accf[b], (uint32_t)((c >> 1) & 1))) { ok = false; return; }
      tc_fence_after();
#pragma unroll
      for (int blk = 0; blk < HW / 32; ++blk) {
        uint32_t r[32];
        const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * BN + h * HW + blk * 32);
        TMEM_LD32(taddr, r);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int j = 0; j < 32; ++j) sum[blk * 32 + j] += __uint_as_float(r[j]);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acce[b]);
    };
    if (nk > 0) fz_load<BN>(xa, xb, ra, rb, kt0, 0, ct, ma0, nc0, Kc);
    for (int i = 0; i < nk && ok; ++i) {
      const int s = i % C::STAGES;
      if (!mbar_wait(&empty[s], (uint32_t)(((i / C::STAGES) & 1) ^ 1))) { ok = false; break; }
      fz_store<THREE, BN>(xa, xb, ra, rb, stage_a_hi(s), stage_a_lo(s), stage_b_hi(s), stage_b_lo(s), ct);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&full[s]);
      if (i + 1 < nk) fz_load<BN>(xa, xb, ra, rb, kt0, i + 1, ct, ma0, nc0, Kc);
      // the previous chunk, once the first stage of the next one is with the tensor core
      if (i % KCH == 0 && i > 0 && ok) { drain(i / KCH - 1); ++drained; }
    }
    while (ok && drained < nchunks) { drain(drained); ++drained; }
    if (!ok && lane == 0) atomicOr(err, DEVERR_TIMEOUT);
    asm volatile("bar.sync 1, %0;" ::"n"(32 * NEPI) : "memory");  // every stage consumed: buffers reusable
    if (partial || epi.scn == 1) {
      constexpr int LDT = BN + 4;
      float* tile = reinterpret_cast<float*>(smem);
      if (ok) {
        float* trow = tile + (q * 32 + lane) * LDT + h * HW;
#pragma unroll
        for (int j = 0; j < HW; j += 4)
          *reinterpret_cast<float4*>(trow + j) = make_float4(sum[j], sum[j + 1], sum[j + 2], sum[j + 3]);
      }
      asm volatile("bar.sync 1, %0;" ::"n"(32 * NEPI) : "memory");
      if (ok) {
        const bool use_beta = (epi.beta.x != 0.f || epi.beta.y != 0.f);
        for (int r = warp - 2; r < BM; r += NEPI) {
          const int grow = m0 + r;
          if (grow >= epi.M) break;
          const float* tr = tile + r * LDT;
          if (partial) {
            float* prow = partial + ((long long)blockIdx.z * epi.M + grow) * (2LL * epi.Nc);
            for (int j = lane; j < BN; j += 32)
              if (n0 + j < 2 * epi.Nc) prow[n0 + j] = tr[j];
          } else {
            float2* crow = epi.C + (long long)grow * epi.scm;
            for (int c = lane; c < BN / 2; c += 32) {
              const int n = n0 / 2 + c;
              if (n < epi.Nc) {
                const float2 a = *reinterpret_cast<const float2*>(tr + 2 * c);
                float2 v;
                v.x = epi.alpha.x * a.x - epi.alpha.y * a.y;
                v.y = epi.alpha.x * a.y + epi.alpha.y * a.x;
                if (use_beta) {
                  const float2 cv = crow[n];
                  v.x += epi.beta.x * cv.x - epi.beta.y * cv.y;
                  v.y += epi.beta.x * cv.y + epi.beta.y * cv.x;
                }
                crow[n] = v;
              }
            }
          }
        }
      }
    } else if (ok && row < epi.M) {
      const int col0 = n0 + h * HW;
      const bool use_beta = (epi.beta.x != 0.f || epi.beta.y != 0.f);
      float2* crow = epi.C + (long long)row * epi.scm;
#pragma unroll
      for (int j = 0; j < HW / 2; ++j) {
        const int n = (col0 >> 1) + j;
        if (n < epi.Nc) {
          const float ar = sum[2 * j], ai = sum[2 * j + 1];
          float2 v;
          v.x = epi.alpha.x * ar - epi.alpha.y * ai;
          v.y = epi.alpha.x * ai + epi.alpha.y * ar;
          float2* p = crow + (long long)n * epi.scn;
          if (use_beta) {
            const float2 cv = *p;
            v.x += epi.beta.x * cv.x - epi.beta.y * cv.y;
            v.y += epi.beta.x * cv.y + epi.beta.y * cv.x;
          }
          *p = v;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    if (nchunks > 0) {
      const int c = nchunks - 1;
      if (!mbar_wait(&accf[c & 1], (uint32_t)((c >> 1) & 1)) && lane == 0) atomicOr(err, DEVERR_TIMEOUT);
    }
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS)
                 : "memory");
  }
}

// ------------------------------------------------------------------ FP64 emulation
// Operand preparation in two passes. Pass 1: the power-of-two exponent E of every row of A'
// (over Re and Im of opA(m, :)) and of every complex column n of opB, E = frexp exponent of
// the largest magnitude, so that |x| 2^-E < 1 (zero rows keep a sentinel below every real
// exponent). Pass 2: the slices d_p = rint(t 2^OZ_BITS), t <- t 2^OZ_BITS - d_p, exact in
// FP64 and in TF32 (|d_p| <= 2^OZ_BITS), written as A'_p / B'^T_p rows in the layout of the
// complex64 path (interleaved Re, Im; the 2 x 2 real embedding for B).
constexpr int OZ_SENT = -(1 << 30);

__device__ __forceinline__ int oz_exp_of(double x) {
  int e = 0;
  (void)frexp(x, &e);
  return x > 0.0 ? e : OZ_SENT;
}

// The slices of x (row exponent e) as integers: N = rint(x 2^(56 - e)) (|N| < 2^56, exact in
// int64), then its balanced base-2^7 digits from the least significant up, d_1..d_7 in
// [-64, 63] and the leading d_0 in [-128, 128]: x 2^-e = sum_p d_p 2^(-7(p+1)) up to half a
// unit of 2^-56. Two FP64 instructions per value (the power-of-two scaling, the conversion)
// instead of a multiply, rint and subtract per slice: B300's FP64 pipe runs at ~1/64 of
// its FP32 rate, and the FP64 form made slicing ~20 % of an emulated complex128 update.
__device__ __forceinline__ void oz_digits(double x, int e, int (&d)[OZ_SLICES]) {
  long long N = 0;
  if (e != OZ_SENT && x != 0.0) {
    const int sh = OZ_SLICES * OZ_BITS - e;
    const int be = 1023 + sh;  // 2^sh as a double when it is a normal number
    const double y = (be >= 1 && be <= 2046) ? x * __longlong_as_double((long long)be << 52) : ldexp(x, sh);
    N = __double2ll_rn(y);
  }
#pragma unroll
  for (int p = OZ_SLICES - 1; p > 0; --p) {
    int r = (int)(N & ((1 << OZ_BITS) - 1));
    if (r >= (1 << (OZ_BITS - 1))) r -= 1 << OZ_BITS;
    d[p] = r;
    N = (N - r) >> OZ_BITS;
  }
  d[0] = (int)N;
}

struct OzJob {
  const double2* src; long long s0, s1; int conj, rows, K;  // rows: M (A) or N (B)
  int* e; __half* out; long long slice_stride; int ld;     // slices in FP16 (exact: |d| <= 128)
  int gx, gy;  // tiles along K and along rows
  int is_b;
};

// pass 1: one 32 x 32 tile; the warps reduce its rows' maxima, one atomic per row and tile
__global__ void k_oz_exp(OzJob a, OzJob b) {
  __shared__ unsigned long long t[32][33];
  pdl_launch_dependents();
  pdl_wait();
  const OzJob& j = blockIdx.z == 0 ? a : b;
  if ((int)blockIdx.x >= j.gx || (int)blockIdx.y >= j.gy) return;
  const int r0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
  // A: element (row m, k) at m s0 + k s1; B: (row n, k) at k s0 + n s1
  const long long srow = j.is_b ? j.s1 : j.s0, sk = j.is_b ? j.s0 : j.s1;
  const bool kc = (sk == 1);
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int rr = kc ? r : threadIdx.x, kk = kc ? threadIdx.x : r;
    const int row = r0 + rr, k = k0 + kk;
    // |x| compared as the integer bit pattern without the sign (monotone for IEEE doubles;
    // a NaN sorts above every number): no FP64 instruction in the pass
    unsigned long long v = 0ull;
    if (row < j.rows && k < j.K) {
      const double2 x = j.src[row * srow + k * sk];
      const unsigned long long a = (unsigned long long)__double_as_longlong(x.x) & 0x7fffffffffffffffull;
      const unsigned long long b = (unsigned long long)__double_as_longlong(x.y) & 0x7fffffffffffffffull;
      v = a > b ? a : b;
    }
    t[rr][kk] = v;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    unsigned long long v = t[r][threadIdx.x];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
      v = w > v ? w : v;
    }
    if (threadIdx.x == 0 && r0 + r < j.rows && v > 0ull)
      atomicMax(j.e + r0 + r, oz_exp_of(__longlong_as_double((long long)v)));
  }
}

// pass 2: slices of one 32 x 32 tile, stores coalesced along K
__global__ void k_oz_slice(OzJob a, OzJob b) {
  __shared__ double2 t[32][33];
  pdl_launch_dependents();
  pdl_wait();
  const OzJob& j = blockIdx.z == 0 ? a : b;
  if ((int)blockIdx.x >= j.gx || (int)blockIdx.y >= j.gy) return;
  const int r0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
  const long long srow = j.is_b ? j.s1 : j.s0, sk = j.is_b ? j.s0 : j.s1;
  const bool kc = (sk == 1);
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int rr = kc ? r : threadIdx.x, kk = kc ? threadIdx.x : r;
    const int row = r0 + rr, k = k0 + kk;
    double2 v = make_double2(0.0, 0.0);
    if (row < j.rows && k < j.K) v = j.src[row * srow + k * sk];
    if (j.conj) v.y = -v.y;
    t[rr][kk] = v;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int row = r0 + r, k = k0 + threadIdx.x;
    if (row >= j.rows || k >= j.K) continue;
    const int e = j.e[row];
    const double2 v = t[r][threadIdx.x];
    int drs[OZ_SLICES], dis[OZ_SLICES];
    oz_digits(v.x, e, drs);
    oz_digits(v.y, e, dis);
#pragma unroll
    for (int p = 0; p < OZ_SLICES; ++p) {
      const float dr = (float)drs[p], di = (float)dis[p];
      __half* o = j.out + (long long)p * j.slice_stride;
      if (!j.is_b) {
        *reinterpret_cast<__half2*>(o + (long long)row * j.ld + 2 * k) = __floats2half2_rn(dr, di);
      } else {
        const long long o0 = (long long)(2 * row) * j.ld + 2 * k;
        *reinterpret_cast<__half2*>(o + o0) = __floats2half2_rn(dr, -di);
        *reinterpret_cast<__half2*>(o + o0 + j.ld) = __floats2half2_rn(di, dr);
      }
    }
  }
}

struct OzEpi {
  double2* C; long long scm, scn;
  double2 alpha, beta;
  int M, Nc;
  const int* ea; const int* eb;
};
struct OzPairs { int n; signed char p[64], q[64]; };

// The GEMM: one 128 x 128 real output tile per CTA, the K loop run once per slice pair
// (A'_p against B'^T_q, fetched by TMA from the stacked slices), the same roles as k_tc_gemm
// (warp 0 TMA, warp 1 TMEM and MMA; here sixteen epilogue warps 2..17). A chunk (CHUNK stages, 128 real K
// terms) never straddles two pairs: its exact FP32 sum is added into FP64 registers with the
// pair's weight, and the rows' and columns' exponents are applied at the end.
constexpr int OZ_BN = 128;
constexpr int OZ_BKH = 64;                   // FP16 elements per stage row (one 128-byte swizzle row)
constexpr int OZ_A_TILE = BM * OZ_BKH * 2;   // 16 KB
constexpr int OZ_B_TILE = OZ_BN * OZ_BKH * 2;
constexpr int OZ_STAGE = OZ_A_TILE + OZ_B_TILE;
constexpr int OZ_STAGES = (192 * 1024) / OZ_STAGE;
constexpr int OZ_SMEM = OZ_STAGES * OZ_STAGE + 1024 + 256;
// instruction descriptor: D fp32, A/B f16 (format 0), both K-major, M = BM, N = OZ_BN
constexpr uint32_t OZ_IDESC = (1u << 4) | ((uint32_t)(OZ_BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
constexpr int OZ_CHUNK = 16;                 // stages per exact FP32 chunk: 16 x 64 = 1024 real K terms
constexpr int OZ_NEPI = 16;                  // epilogue warps: four lane quarters x four column quarters
constexpr int OZ_NT = 64 + 32 * OZ_NEPI;
// TMEM: the two chunk accumulators in columns [0, 2 OZ_BN), the FP64 level sums above them
// (each epilogue thread's 32 doubles as 64 words of its own lane: one double per output)
constexpr int OZ_TMEM_COLS = 512;
constexpr int OZ_ACC64_COL = 2 * OZ_BN;
static_assert(OZ_ACC64_COL + 4 * 2 * (OZ_BN / 4) <= OZ_TMEM_COLS, "FP64 sums in TMEM");

__global__ void __launch_bounds__(OZ_NT, 1)
    k_oz_gemm(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB, OzEpi epi,
              int Kp, int a_rows, int b_rows, OzPairs pr, double2* part, unsigned* err) {
  // grid.z > 1 splits the slice pairs over CTAs (products with few output tiles): CTA z takes
  // pairs [p_lo, p_hi) and writes its scaled partial tile to part[z] for k_oz_sum
  static_assert(BM * (OZ_BN / 2 + 1) * 16 <= OZ_STAGES * OZ_STAGE, "staged epilogue tile");
  constexpr int HW = OZ_BN / 4;  // real columns per epilogue thread (four column quarters)
  pdl_launch_dependents();
  pdl_wait();
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = smem_raw + ((1024 - (s_u32(smem_raw) & 1023)) & 1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + OZ_STAGES * OZ_STAGE);
  uint64_t* empty = full + OZ_STAGES;
  uint64_t* accf = empty + OZ_STAGES;
  uint64_t* acce = accf + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acce + 2);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n0 = blockIdx.x * OZ_BN, m0 = blockIdx.y * BM;
  const int nk = (Kp + OZ_BKH - 1) / OZ_BKH;
  const int cpp = (nk + OZ_CHUNK - 1) / OZ_CHUNK;  // chunks per pair
  const int per_z = (pr.n + (int)gridDim.z - 1) / (int)gridDim.z;
  const int p_lo = min(pr.n, (int)blockIdx.z * per_z), p_hi = min(pr.n, p_lo + per_z);
  const int npairs = p_hi - p_lo;
  const int total = npairs * nk;
  const int nchunks = npairs * cpp;
  if (threadIdx.x == 0) {
    for (int st = 0; st < OZ_STAGES; ++st) { mbar_init(&full[st], 1); mbar_init(&empty[st], 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(&accf[b], 1); mbar_init(&acce[b], OZ_NEPI); }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_u32(tmem_slot)),
                 "r"(OZ_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  auto stage_a = [&](int st) { return smem + st * OZ_STAGE; };
  auto stage_b = [&](int st) { return smem + st * OZ_STAGE + OZ_A_TILE; };

  if (warp == 0) {
    if (lane == 0) {
      bool ok = true;
      int issued = 0;
      for (int it = 0; it < total && ok; ++it) {
        const int st = it % OZ_STAGES;
        const uint32_t ph = (uint32_t)((it / OZ_STAGES) & 1);
        if (!mbar_wait(&empty[st], ph ^ 1u)) { ok = false; break; }
        const int p = p_lo + it / nk, i = it % nk;
        mbar_expect_tx(&full[st], OZ_STAGE);
        tma_load(stage_a(st), &tA, &full[st], i * OZ_BKH, pr.p[p] * a_rows + m0);
        tma_load(stage_b(st), &tB, &full[st], i * OZ_BKH, pr.q[p] * b_rows + n0);
        ++issued;
      }
      if (!ok) atomicOr(err, DEVERR_TIMEOUT);
      for (int it = (issued > OZ_STAGES ? issued - OZ_STAGES : 0); it < issued; ++it) {
        if (!mbar_wait(&full[it % OZ_STAGES], (uint32_t)((it / OZ_STAGES) & 1))) {
          atomicOr(err, DEVERR_TIMEOUT);
          break;
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      bool ok = true;
      for (int c = 0; c < nchunks && ok; ++c) {
        const int b = c & 1;
        if (c >= 2 && !mbar_wait(&acce[b], (uint32_t)(((c >> 1) - 1) & 1))) { ok = false; break; }
        tc_fence_after();
        const uint32_t acc_t = tmem + (uint32_t)(b * OZ_BN);
        const int pl = c / cpp, kc = c % cpp;  // pair p_lo + pl
        const int i0 = kc * OZ_CHUNK, i1 = min(nk, i0 + OZ_CHUNK);
        for (int i = i0; i < i1; ++i) {
          const int it = pl * nk + i;
          const int st = it % OZ_STAGES;
          if (!mbar_wait(&full[st], (uint32_t)((it / OZ_STAGES) & 1))) { ok = false; break; }
          tc_fence_after();
          const uint32_t a0 = s_u32(stage_a(st)), b0 = s_u32(stage_b(st));
#pragma unroll
          for (int k = 0; k < OZ_BKH / 16; ++k) {
            const uint32_t off = k * 32;  // 16 f16 = 32 bytes along K inside the swizzle row
            tc_mma_f16(acc_t, desc_sw128(a0 + off), desc_sw128(b0 + off), OZ_IDESC, (i > i0 || k > 0) ? 1u : 0u);
          }
          tc_commit(&empty[st]);
        }
        tc_commit(&accf[b]);
      }
      if (!ok) atomicOr(err, DEVERR_TIMEOUT);
    }
  } else {
    const int q = warp & 3;
    const int h = (warp - 2) >> 2;  // column quarter
    const int row = m0 + q * 32 + lane;
    // Each chunk is an exact integer of at most 2^24 in magnitude, added into FP64 registers
    // with its pair's power-of-two weight (one DFMA per element and chunk of 1024 K terms).
    // Chunks of one weight level (p + q; the pairs come ordered by level) are exact integers
    // of at most 2^24 in magnitude: they are summed exactly in int32 (at most 127 chunks per
    // flush), and only a finished level sum is added into the FP64 registers with its weight
    // 2^(-OZ_BITS (p+q+2)). The FP64 pipe, much narrower than the tensor core's chunk rate,
    // then does one FMA per element and level instead of one per chunk.
    // The FP64 sums live in TMEM (this thread's lane, columns OZ_ACC64_COL + 2 HW h ..): held
    // in registers beside the int32 level sums they spilled to local memory. A flush loads
    // them, adds the level and stores them back; they return to registers only at the end.
    int iacc[HW];
#pragma unroll
    for (int jj = 0; jj < HW; ++jj) iacc[jj] = 0;
    const uint32_t t64 = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(OZ_ACC64_COL + 2 * HW * h);
    {
      uint32_t z[32];
#pragma unroll
      for (int jj = 0; jj < 32; ++jj) z[jj] = 0u;
#pragma unroll
      for (int blk = 0; blk < 2 * HW / 32; ++blk) TMEM_ST32(t64 + blk * 32, z);
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    int lvl = -1, nin = 0;
    auto flush = [&]() {
      if (lvl >= 0 && nin > 0) {
        const double w = ldexp(1.0, -OZ_BITS * (lvl + 2));
#pragma unroll
        for (int blk = 0; blk < 2 * HW / 32; ++blk) {
          uint32_t r[32];
          TMEM_LD32(t64 + blk * 32, r);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) {
            double a = __hiloint2double((int)r[2 * jj + 1], (int)r[2 * jj]);
            a = fma((double)iacc[blk * 16 + jj], w, a);
            iacc[blk * 16 + jj] = 0;
            r[2 * jj] = (uint32_t)__double2loint(a);
            r[2 * jj + 1] = (uint32_t)__double2hiint(a);
          }
          TMEM_ST32(t64 + blk * 32, r);
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      }
      nin = 0;
    };
    bool ok = true;
    for (int c = 0; c < nchunks; ++c) {
      const int b = c & 1;
      if (!mbar_wait(&accf[b], (uint32_t)((c >> 1) & 1))) { ok = false; break; }
      tc_fence_after();
      const int p = p_lo + c / cpp;
      const int l = pr.p[p] + pr.q[p];
      if (l != lvl || nin == 127) { flush(); lvl = l; }
#pragma unroll
      for (int blk = 0; blk < HW / 16; ++blk) {
        uint32_t r[16];
        const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * OZ_BN + h * HW + blk * 16);
        TMEM_LD16(taddr, r);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) iacc[blk * 16 + jj] += __float2int_rn(__uint_as_float(r[jj]));
      }
      ++nin;
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acce[b]);
    }
    flush();
    if (!ok && lane == 0) atomicOr(err, DEVERR_TIMEOUT);
    double acc[HW];
#pragma unroll
    for (int blk = 0; blk < 2 * HW / 32; ++blk) {
      uint32_t r[32];
      TMEM_LD32(t64 + blk * 32, r);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int jj = 0; jj < 16; ++jj) acc[blk * 16 + jj] = __hiloint2double((int)r[2 * jj + 1], (int)r[2 * jj]);
    }
    auto sum = [&](int jj) { return acc[jj]; };
    const bool use_beta = (epi.beta.x != 0.0 || epi.beta.y != 0.0);
    const int ea = (row < epi.M) ? epi.ea[row] : OZ_SENT;
    if (part) {
      // this CTA's share of the pairs, exponents applied, into its partial tile
      if (ok && row < epi.M) {
        const int col0 = n0 + h * HW;
        double2* prow = part + ((long long)blockIdx.z * epi.M + row) * epi.Nc;
#pragma unroll
        for (int jj = 0; jj < HW / 2; ++jj) {
          const int n = (col0 >> 1) + jj;
          if (n < epi.Nc) {
            const int eb = epi.eb[n];
            const bool z = (ea == OZ_SENT || eb == OZ_SENT);
            prow[n] = z ? make_double2(0.0, 0.0)
                        : make_double2(ldexp(sum(2 * jj), ea + eb), ldexp(sum(2 * jj + 1), ea + eb));
          }
        }
      }
    } else if (epi.scn == 1) {
      // stage the tile (complex128 results, row exponents applied) in the idle pipeline
      // buffers, then each warp writes whole row segments
      constexpr int LDT = OZ_BN / 2 + 1;  // complex values per staged row (odd: no bank conflicts)
      double2* tile = reinterpret_cast<double2*>(smem);
      if (ok) {
        double2* trow = tile + (q * 32 + lane) * LDT + h * (HW / 2);
#pragma unroll
        for (int jj = 0; jj < HW / 2; ++jj)
          trow[jj] = ea == OZ_SENT ? make_double2(0.0, 0.0)
                                   : make_double2(ldexp(sum(2 * jj), ea), ldexp(sum(2 * jj + 1), ea));
      }
      asm volatile("bar.sync 1, %0;" ::"n"(32 * OZ_NEPI) : "memory");
      if (ok) {
        for (int r = warp - 2; r < BM; r += OZ_NEPI) {
          const int grow = m0 + r;
          if (grow >= epi.M) break;
          const double2* tr = tile + r * LDT;
          double2* crow = epi.C + (long long)grow * epi.scm;
          for (int cc = lane; cc < OZ_BN / 2; cc += 32) {
            const int n = n0 / 2 + cc;
            if (n < epi.Nc) {
              const int eb = epi.eb[n];
              const double2 a = eb == OZ_SENT ? make_double2(0.0, 0.0)
                                              : make_double2(ldexp(tr[cc].x, eb), ldexp(tr[cc].y, eb));
              double2 v;
              v.x = epi.alpha.x * a.x - epi.alpha.y * a.y;
              v.y = epi.alpha.x * a.y + epi.alpha.y * a.x;
              if (use_beta) {
                const double2 cv = crow[n];
                v.x += epi.beta.x * cv.x - epi.beta.y * cv.y;
                v.y += epi.beta.x * cv.y + epi.beta.y * cv.x;
              }
              crow[n] = v;
            }
          }
        }
      }
    } else if (ok && row < epi.M) {
      const int col0 = n0 + h * HW;
      double2* crow = epi.C + (long long)row * epi.scm;
#pragma unroll
      for (int jj = 0; jj < HW / 2; ++jj) {
        const int n = (col0 >> 1) + jj;
        if (n < epi.Nc) {
          const int eb = epi.eb[n];
          const bool z = (ea == OZ_SENT || eb == OZ_SENT);
          const double ar = z ? 0.0 : ldexp(sum(2 * jj), ea + eb), ai = z ? 0.0 : ldexp(sum(2 * jj + 1), ea + eb);
          double2 v;
          v.x = epi.alpha.x * ar - epi.alpha.y * ai;
          v.y = epi.alpha.x * ai + epi.alpha.y * ar;
          double2* pp = crow + (long long)n * epi.scn;
          if (use_beta) {
            const double2 cv = *pp;
            v.x += epi.beta.x * cv.x - epi.beta.y * cv.y;
            v.y += epi.beta.x * cv.y + epi.beta.y * cv.x;
          }
          *pp = v;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    if (nchunks > 0) {
      const int c = nchunks - 1;
      if (!mbar_wait(&accf[c & 1], (uint32_t)((c >> 1) & 1)) && lane == 0) atomicOr(err, DEVERR_TIMEOUT);
    }
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(OZ_TMEM_COLS) : "memory");
  }
}

// C = alpha sum_z part[z] + beta C for a pair-split emulated product (part: splits x M x N)
__global__ void k_oz_sum(const double2* part, int splits, OzEpi epi) {
  pdl_launch_dependents();
  pdl_wait();
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long MN = (long long)epi.M * epi.Nc;
  if (idx >= MN) return;
  const int m = (int)(idx / epi.Nc), n = (int)(idx % epi.Nc);
  double ar = 0.0, ai = 0.0;
  for (int z = 0; z < splits; ++z) {
    const double2 v = part[(long long)z * MN + idx];
    ar += v.x; ai += v.y;
  }
  double2 v;
  v.x = epi.alpha.x * ar - epi.alpha.y * ai;
  v.y = epi.alpha.x * ai + epi.alpha.y * ar;
  double2* c = epi.C + (long long)m * epi.scm + (long long)n * epi.scn;
  if (epi.beta.x != 0.0 || epi.beta.y != 0.0) {
    const double2 cv = *c;
    v.x += epi.beta.x * cv.x - epi.beta.y * cv.y;
    v.y += epi.beta.x * cv.y + epi.beta.y * cv.x;
  }
  *c = v;
}

// ------------------------------------------------------------------ host
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

int get_encode() {
  std::call_once(g_encode_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  });
  if (!g_encode) { set_last_message("cuTensorMapEncodeTiled unavailable"); return QRTEBD_ERR_CUDA; }
  return QRTEBD_OK;
}

int make_map(CUtensorMap* tm, const float* base, int rows, int cols, int ld, int box_rows) {
  cuuint64_t gdim[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t gstride[1] = {(cuuint64_t)ld * 4};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), gdim,
                        gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) { set_last_message("cuTensorMapEncodeTiled failed"); return QRTEBD_ERR_CUDA; }
  return QRTEBD_OK;
}

inline int ld_for(int k) { return (int)align_up((size_t)2 * k, 32); }
// FP16 slice rows: 2k halves padded to whole 128-byte rows
inline int ld_for_h(int k) { return (int)align_up((size_t)2 * k, 64); }

int make_map_h(CUtensorMap* tm, const __half* base, int rows, int cols, int ld, int box_rows) {
  cuuint64_t gdim[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t gstride[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)OZ_BKH, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<__half*>(base), gdim,
                        gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) { set_last_message("cuTensorMapEncodeTiled failed"); return QRTEBD_ERR_CUDA; }
  return QRTEBD_OK;
}

template <bool THREE, int BN> int set_attrs_once() {
  static std::once_flag once;
  static cudaError_t e = cudaSuccess;
  std::call_once(once, [] {
    e = cudaFuncSetAttribute(k_tc_gemm<THREE, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             Cfg<THREE, BN>::SMEM);
  });
  QR_CUDA_TRY(e);
  return QRTEBD_OK;
}

template <bool THREE, int BN>
int launch_tc(dim3 grid, cudaStream_t st, const CUtensorMap& a_hi, const CUtensorMap& a_lo,
              const CUtensorMap& b_hi, const CUtensorMap& b_lo, const Epi& e, int Kp, int per,
              float* part, int m_off, unsigned* err, int ktri) {
  QR_TRY((set_attrs_once<THREE, BN>()));
  QR_CUDA_TRY(launch_pdl(k_tc_gemm<THREE, BN>, grid, dim3(NTHREADS), Cfg<THREE, BN>::SMEM, st, a_hi,
                         a_lo, b_hi, b_lo, e, Kp, per, part, m_off, err, ktri));
  return QRTEBD_OK;
}

template <bool THREE, int BN> int set_fz_attrs_once() {
  static std::once_flag once;
  static cudaError_t e = cudaSuccess;
  std::call_once(once, [] {
    e = cudaFuncSetAttribute(k_tc_gemm_fz<THREE, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             Cfg<THREE, BN>::SMEM);
  });
  QR_CUDA_TRY(e);
  return QRTEBD_OK;
}

template <bool THREE, int BN>
int launch_fz(dim3 grid, cudaStream_t st, const RawOp& ra, const RawOp& rb, const Epi& e, int per, float* part,
              int m_off, unsigned* err) {
  QR_TRY((set_fz_attrs_once<THREE, BN>()));
  QR_CUDA_TRY(launch_pdl(k_tc_gemm_fz<THREE, BN>, grid, dim3(NTHREADS), Cfg<THREE, BN>::SMEM, st, ra, rb, e,
                         per, part, m_off, err));
  return QRTEBD_OK;
}

// Operand preparation as a separate pass (1, the default) or inside the GEMM kernel (0)
std::atomic<int> g_prep_mode{1};

// The in-kernel preparation reads pairs of complex values with 16-byte loads: an operand
// qualifies when it is contiguous along K or along its other index, the other stride is
// even and the base is 16-byte aligned.
// The vector form of the separate preparation: contiguous along K, the other stride even
// and the base 16-byte aligned, so that every pair of K is one aligned 16-byte load.
bool vec_layout(const float2* p, long long s_rows, long long s_k) {
  return s_k == 1 && s_rows % 2 == 0 && (reinterpret_cast<uintptr_t>(p) & 15) == 0;
}

bool raw_layout(const float2* p, long long s_rows, long long s_k, bool is_b, int* kmajor) {
  // A: (m, k) at p[m s_rows + k s_k]; B: (k, n) at p[k s_k + n s_rows]
  if ((reinterpret_cast<uintptr_t>(p) & 15) != 0) return false;
  if (s_k == 1 && s_rows % 2 == 0) { *kmajor = 1; return true; }
  if (s_rows == 1 && s_k % 2 == 0) { *kmajor = 0; return true; }
  (void)is_b;
  return false;
}

// tuning table and the recording pass
std::mutex g_tune_mu;
std::map<TcShape, TcTuned> g_tune;
bool g_recording = false;
std::vector<TcShape> g_recorded;

}  // namespace

void tc_carve(Arena& ar, int max_m, int max_k, int max_n, TcWorkspace& w) {
  size_t ld = (size_t)ld_for(max_k);
  w.a_cap = (size_t)max_m * ld;
  w.b_cap = (size_t)2 * max_n * ld;
  for (int i = 0; i < 2; ++i) {
    w.a[i] = TcSlot{};
    w.a[i].hi = ar.take<float>(w.a_cap);
    w.a[i].lo = ar.take<float>(w.a_cap);
  }
  w.b = TcSlot{};
  w.b.hi = ar.take<float>(w.b_cap);
  w.b.lo = ar.take<float>(w.b_cap);
  w.p_cap = (size_t)1 << 23;  // 32 MB of split-K partial sums
  w.partial = ar.take<float>(w.p_cap);
}

int tc_prep_mode(int mode) { return g_prep_mode.exchange(mode); }

void tc_invalidate(TcWorkspace& w) {
  w.a[0].valid = w.a[1].valid = false;
  w.b.valid = false;
}

bool tc_gemm_eligible(const GemmArgs<float>& g) {
  // K < 64: two K-blocks or fewer, where the operand preparation and the fixed cost of
  // the tensor-core kernel outweigh the CUDA-core GEMM (measured 2x slower at K = 32)
  return g.batch == 1 && std::max(g.M, g.N) >= 128 && std::min(g.M, g.N) >= 16 && g.K >= 64 &&
         (double)g.M * g.N * g.K >= (double)(1 << 21);
}

int tc_gemm(const GemmArgs<float>& g0, bool three, TcWorkspace& w, cudaStream_t st, int prof_family) {
  return tc_gemm_cfg(g0, three, w, st, nullptr, prof_family);
}

int tc_gemm_cfg(const GemmArgs<float>& g0, bool three, TcWorkspace& w, cudaStream_t st,
                const TcConfig* force, int prof_family) {
  // C = A B with N > M is run as C^T = B^T A^T: the tile is 128 rows tall, and the
  // B operand is the one stored twice over (2x2 real embedding), so it should be the
  // smaller one
  GemmArgs<float> g = g0;
  bool cacheable = g0.reuse_a;
  // a lower-triangular A limits each tile row's K, an upper-triangular B each tile column's;
  // the swap below exchanges the two
  const bool swap = g0.N > g0.M;
  const int ktri = g0.tri_a ? (swap ? 2 : 1) : g0.tri_b ? (swap ? 1 : 2) : 0;
  if (g0.N > g0.M) {
    cacheable = false;
    g.M = g0.N; g.N = g0.M;
    g.A = g0.B; g.sam = g0.sbn; g.sak = g0.sbk; g.conj_a = g0.conj_b;
    g.B = g0.A; g.sbk = g0.sak; g.sbn = g0.sam; g.conj_b = g0.conj_a;
    g.scm = g0.scn; g.scn = g0.scm;
  }
  const int M = g.M, N = g.N, K = g.K;
  const int ld = ld_for(K);
  if ((size_t)M * ld > w.a_cap || (size_t)2 * N * ld > w.b_cap || !w.a[0].hi || !w.b.hi)
    return gemm_simt<float>(g0, st, nullptr, 0, prof_family == PROF_TC_GEMM ? PROF_SIMT_GEMM : prof_family);
  QR_TRY(get_encode());
  const TcShape key{M, N, K, three ? 1 : 0};
  TcConfig cfg;
  bool have = false;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (g_recording) g_recorded.push_back(key);
    if (force) { cfg = *force; have = true; }
    else if (concurrency() == 1) {
      // the table holds each shape's best configuration when the product runs alone;
      // beside other bond updates the heuristic one (256-column tiles, K-splits for the
      // product's share of the SMs) measured faster
      auto it = g_tune.find(key);
      if (it != g_tune.end()) { cfg = it->second.cfg; have = true; }
    }
  }
  const int bn = (have && cfg.bn == 128) ? 128 : 256;
  // Operand preparation inside the GEMM kernel where the layouts allow, for 128-column
  // tiles only (register budget); otherwise A' and B'^T in one separate launch. A' of an
  // operand marked for reuse lives in slot 0, which no other operand overwrites, so it
  // survives the GEMMs in between (the QR's); every other A' goes to slot 1
  int a_km = 0, b_km = 0;
  const bool fused = bn == 128 && g_prep_mode.load() == 0 && raw_layout(g.A, g.sam, g.sak, false, &a_km) &&
                     raw_layout(g.B, g.sbn, g.sbk, true, &b_km);
  TcSlot* sa = nullptr;
  if (cacheable) {
    TcSlot& s = w.a[0];
    if (s.valid && s.src == g.A && s.s0 == g.sam && s.s1 == g.sak && s.rows == M && s.cols == K &&
        s.conj == g.conj_a && s.three == three && s.ld == ld)
      sa = &s;
  }
  const bool need_a = !fused && (sa == nullptr);
  if (sa == nullptr) sa = &w.a[cacheable ? 0 : 1];
  if (!fused) {
    PrepJob ja{g.A, g.sam, g.sak, g.conj_a ? 1 : 0, M, K, sa->hi, sa->lo, ld,
               need_a ? (int)ceil_div(K, 32) : 0, need_a ? (int)ceil_div(M, 32) : 0, 0};
    PrepJob jb{g.B, g.sbk, g.sbn, g.conj_b ? 1 : 0, N, K, w.b.hi, w.b.lo, ld,
               (int)ceil_div(K, 32), (int)ceil_div(N, 32), 0};
    // the vector form where the operand runs along K in 16-byte aligned pairs
    const long long kp = (K + 1) / 2;
    ja.vec = need_a && vec_layout(g.A, g.sam, g.sak) && (long long)M * kp < (1LL << 31);
    jb.vec = vec_layout(g.B, g.sbn, g.sbk) && (long long)N * kp < (1LL << 31);
    // grid: the tile form's tiles; a vector-form operand wants about two units per thread
    // on at most 8 blocks per SM (its blocks grid-stride over the rest), laid over the
    // tile form's rows of blocks when the other operand has some
    unsigned gx = 1, gy = 1;
    for (const PrepJob* j : {&ja, &jb})
      if (!j->vec) { gx = std::max(gx, (unsigned)j->gx); gy = std::max(gy, (unsigned)j->gy); }
    for (const PrepJob* j : {&ja, &jb})
      if (j->vec) {
        const long long blocks = std::min<long long>(ceil_div((long long)j->rows * kp, 512), 148 * 8);
        gx = std::max(gx, (unsigned)ceil_div(blocks, (long long)gy));
      }
    dim3 grid(gx, gy, 2);
    ProfScope prof(PROF_PREP, st, 0,
                   (need_a ? 8.0 * M * K + (three ? 16.0 : 8.0) * M * K : 0.0) +
                       8.0 * N * K + (three ? 32.0 : 16.0) * N * K);
    QR_CUDA_TRY(launch_pdl(k_prep, grid, dim3(32, 8), 0, st, ja, jb, three ? 1 : 0));
    note_launch();
  }
  if (need_a) {
    sa->valid = cacheable; sa->src = g.A; sa->s0 = g.sam; sa->s1 = g.sak; sa->rows = M; sa->cols = K;
    sa->conj = g.conj_a; sa->three = three; sa->ld = ld;
  }
  CUtensorMap ta_hi, ta_lo, tb_hi, tb_lo;
  if (!fused) {
    QR_TRY(make_map(&ta_hi, sa->hi, M, 2 * K, ld, BM));
    QR_TRY(make_map(&ta_lo, three ? sa->lo : sa->hi, M, 2 * K, ld, BM));
    QR_TRY(make_map(&tb_hi, w.b.hi, 2 * N, 2 * K, ld, bn));
    QR_TRY(make_map(&tb_lo, three ? w.b.lo : w.b.hi, 2 * N, 2 * K, ld, bn));
  }
  const RawOp ra{g.A, g.sam, g.sak, g.conj_a ? 1 : 0, a_km, M, K};
  const RawOp rb{g.B, g.sbk, g.sbn, g.conj_b ? 1 : 0, b_km, N, K};

  Epi epi{g.C, g.scm, g.scn, g.alpha, g.beta, M, N};
  const int nx = (int)ceil_div(2LL * N, bn), ny = (int)ceil_div(M, BM);
  const int nk = (int)ceil_div(2LL * K, BK);
  // beside n - 1 other bond updates a product sizes its K-splits for its share of the SMs,
  // and runs no tail split (other updates' kernels fill the SMs a short last wave leaves)
  const int conc = force ? 1 : concurrency();
  const int nsm = conc > 1 ? std::max(1, 148 / conc) : 148;
  unsigned* err = device_error_word();
  // one launch over tile rows [ty0, ty0 + nty) with `splits` K-splits (then their sum)
  auto run = [&](int ty0, int nty, int splits) -> int {
    const int per = (int)ceil_div(nk, splits);
    splits = (int)ceil_div(nk, per);
    const int m_off = ty0 * BM;
    Epi e = epi;
    e.C = epi.C + (long long)m_off * epi.scm;
    e.M = std::min(M, (ty0 + nty) * BM) - m_off;
    float* part = splits > 1 ? w.partial : nullptr;
    dim3 grid((unsigned)nx, (unsigned)nty, (unsigned)splits);
    {
      ProfScope prof(prof_family, st, 8.0 * e.M * N * K);
      if (fused) {
        if (three) QR_TRY((launch_fz<true, 128>(grid, st, ra, rb, e, per, part, m_off, err)));
        else QR_TRY((launch_fz<false, 128>(grid, st, ra, rb, e, per, part, m_off, err)));
      } else if (three && bn == 256)
        QR_TRY((launch_tc<true, 256>(grid, st, ta_hi, ta_lo, tb_hi, tb_lo, e, 2 * K, per, part, m_off, err, ktri)));
      else if (three)
        QR_TRY((launch_tc<true, 128>(grid, st, ta_hi, ta_lo, tb_hi, tb_lo, e, 2 * K, per, part, m_off, err, ktri)));
      else if (bn == 256)
        QR_TRY((launch_tc<false, 256>(grid, st, ta_hi, ta_lo, tb_hi, tb_lo, e, 2 * K, per, part, m_off, err, ktri)));
      else
        QR_TRY((launch_tc<false, 128>(grid, st, ta_hi, ta_lo, tb_hi, tb_lo, e, 2 * K, per, part, m_off, err, ktri)));
      note_launch();
      QR_CUDA_TRY(cudaGetLastError());
    }
    if (splits > 1) {
      QR_CUDA_TRY(launch_pdl(k_splitk_sum, dim3((unsigned)ceil_div((long long)e.M * N, 256)), dim3(256),
                             0, st, static_cast<const float*>(part), splits, e));
      note_launch();
      QR_CUDA_TRY(cudaGetLastError());
    }
    return QRTEBD_OK;
  };
  auto fit_splits = [&](int splits, long long rows) {
    splits = std::max(1, std::min(splits, std::min(nk, 32)));
    while (splits > 1 && (size_t)splits * rows * 2 * N > w.p_cap) --splits;
    return splits;
  };
  const int tiles = nx * ny;
  if (have && cfg.splits > 1) return run(0, ny, fit_splits(cfg.splits, M));
  if (!(have && cfg.splits == 1) && tiles < 100 && nk >= 2 * CHUNK) {
    // split K when the tile grid leaves most SMs idle
    int splits = std::min<int>((int)ceil_div(nsm, tiles), nk / CHUNK);
    return run(0, ny, fit_splits(splits, M));
  }
  if (conc == 1 && (!have || cfg.tail) && tiles > nsm && nk >= 4 * CHUNK) {
    // a last wave of a few tiles would leave most SMs idle for a whole tile's time: run the
    // full waves, then the remaining tile rows with their K split over the idle SMs
    const int tail_rows = (int)ceil_div(tiles % nsm, nx);
    const int tail_tiles = tail_rows * nx;
    if (tail_rows > 0 && tail_rows < ny && tail_tiles <= nsm / 3) {
      const int ts = fit_splits(std::min(nsm / tail_tiles, nk / CHUNK), (long long)tail_rows * BM);
      if (ts >= 2) {
        QR_TRY(run(0, ny - tail_rows, 1));
        return run(ny - tail_rows, tail_rows, ts);
      }
    }
  }
  return run(0, ny, 1);
}

// ------------------------------------------------------------------ autotuner
namespace {
__global__ void k_fill_test(float2* x, long long n, unsigned seed) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  unsigned h = (unsigned)i * 2654435761u ^ seed;
  h ^= h >> 15; h *= 2246822519u; h ^= h >> 13;
  x[i] = make_float2((float)(h & 0xffff) / 32768.f - 1.f, (float)(h >> 16) / 32768.f - 1.f);
}
}  // namespace

void oz_carve(Arena& ar, int max_m, int max_k, int max_n, OzWorkspace& w) {
  const size_t ld = (size_t)ld_for_h(max_k);
  w.a_cap = (size_t)OZ_SLICES * max_m * ld;
  w.b_cap = (size_t)OZ_SLICES * 2 * max_n * ld;
  w.ea_cap = (size_t)max_m;
  w.eb_cap = (size_t)max_n;
  w.a = ar.take<unsigned short>(w.a_cap);
  w.b = ar.take<unsigned short>(w.b_cap);
  w.ea = ar.take<int>(w.ea_cap);
  w.eb = ar.take<int>(w.eb_cap);
  w.part_cap = (size_t)1 << 21;  // 32 MB of pair-split partial tiles (complex128)
  w.part = ar.take<double2>(w.part_cap);
}

bool oz_gemm_eligible(const GemmArgs<double>& g) {
  // products with enough work to amortise the slicing: at least 64 output tiles, or fewer
  // tiles with a long K whose slice pairs are split over CTAs; the rest stay on the FP64
  // CUDA cores
  const long long mm = std::max(g.M, g.N), nn = std::min(g.M, g.N);
  if (g.batch != 1 || g.K < 64) return false;
  const long long tiles = ceil_div(mm, BM) * ceil_div(2 * nn, OZ_BN);
  return tiles >= 64 || (g.K >= 512 && (double)g.M * g.N * g.K >= (double)(1 << 25));
}

int oz_gemm(const GemmArgs<double>& g0, OzWorkspace& w, cudaStream_t st, int prof_family) {
  // as the complex64 path: C = A B with N > M runs as C^T = B^T A^T
  GemmArgs<double> g = g0;
  if (g0.N > g0.M) {
    g.M = g0.N; g.N = g0.M;
    g.A = g0.B; g.sam = g0.sbn; g.sak = g0.sbk; g.conj_a = g0.conj_b;
    g.B = g0.A; g.sbk = g0.sak; g.sbn = g0.sam; g.conj_b = g0.conj_a;
    g.scm = g0.scn; g.scn = g0.scm;
  }
  const int M = g.M, N = g.N, K = g.K;
  if (M <= 0 || N <= 0) return QRTEBD_OK;
  const int ld = ld_for_h(K);
  if (K <= 0 || (size_t)OZ_SLICES * M * ld > w.a_cap || (size_t)OZ_SLICES * 2 * N * ld > w.b_cap ||
      (size_t)M > w.ea_cap || (size_t)N > w.eb_cap || !w.a || !w.b)
    return gemm_simt<double>(g0, st, nullptr, 0, prof_family == PROF_TC_GEMM ? PROF_SIMT_GEMM : prof_family);
  QR_TRY(get_encode());
  // exponents (memset 0x80 bytes: a sentinel below every exponent), then the slices
  QR_CUDA_TRY(cudaMemsetAsync(w.ea, 0x80, (size_t)M * sizeof(int), st));
  QR_CUDA_TRY(cudaMemsetAsync(w.eb, 0x80, (size_t)N * sizeof(int), st));
  __half* sa = reinterpret_cast<__half*>(w.a);
  __half* sb = reinterpret_cast<__half*>(w.b);
  OzJob ja{g.A, g.sam, g.sak, g.conj_a ? 1 : 0, M, K, w.ea, sa, (long long)M * ld, ld,
           (int)ceil_div(K, 32), (int)ceil_div(M, 32), 0};
  OzJob jb{g.B, g.sbk, g.sbn, g.conj_b ? 1 : 0, N, K, w.eb, sb, (long long)2 * N * ld, ld,
           (int)ceil_div(K, 32), (int)ceil_div(N, 32), 1};
  {
    dim3 grid((unsigned)std::max(ja.gx, jb.gx), (unsigned)std::max(ja.gy, jb.gy), 2);
    ProfScope prof(PROF_PREP, st, 0, 16.0 * (M + N) * (double)K * 2 + 2.0 * OZ_SLICES * 2 * K * ((double)M + 2.0 * N));
    QR_CUDA_TRY(launch_pdl(k_oz_exp, grid, dim3(32, 8), 0, st, ja, jb));
    note_launch();
    QR_CUDA_TRY(launch_pdl(k_oz_slice, grid, dim3(32, 8), 0, st, ja, jb));
    note_launch();
  }
  // the slices of every operand stacked as one tensor: slice p's rows start at p * rows
  CUtensorMap ta, tb;
  QR_TRY(make_map_h(&ta, sa, OZ_SLICES * M, 2 * K, ld, BM));
  QR_TRY(make_map_h(&tb, sb, OZ_SLICES * 2 * N, 2 * K, ld, OZ_BN));
  // the slice pairs p + q <= OZ_SLICES - 1, ordered by level p + q (the kernel sums a level's
  // chunks in integers before one FP64 add)
  OzPairs pr{};
  for (int l = 0; l <= OZ_SLICES - 1; ++l)
    for (int p = 0; p <= l; ++p) { pr.p[pr.n] = (signed char)p; pr.q[pr.n] = (signed char)(l - p); ++pr.n; }
  OzEpi epi{g.C, g.scm, g.scn, make_double2(g.alpha.x, g.alpha.y), make_double2(g.beta.x, g.beta.y), M, N,
            w.ea, w.eb};
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(once, [] { attr_err = cudaFuncSetAttribute(k_oz_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM); });
  QR_CUDA_TRY(attr_err);
  const int nx = (int)ceil_div(2LL * N, OZ_BN), ny = (int)ceil_div(M, BM);
  // few output tiles: split the slice pairs over CTAs (as many groups as fill the SMs, within
  // the partial-tile buffer), then sum the partial tiles
  int splits = 1;
  if (nx * ny < 148 && w.part) {
    splits = std::min<int>(pr.n, (int)ceil_div(148, nx * ny));
    while (splits > 1 && (size_t)splits * M * N > w.part_cap) --splits;
  }
  dim3 grid((unsigned)nx, (unsigned)ny, (unsigned)splits);
  {
    // algorithmic work: the complex product (8 M N K real flops), as for every GEMM family
    ProfScope prof(prof_family, st, 8.0 * M * N * K);
    QR_CUDA_TRY(launch_pdl(k_oz_gemm, grid, dim3(OZ_NT), OZ_SMEM, st, ta, tb, epi, 2 * K, M, 2 * N, pr,
                           splits > 1 ? w.part : static_cast<double2*>(nullptr), device_error_word()));
    note_launch();
    QR_CUDA_TRY(cudaGetLastError());
  }
  if (splits > 1) {
    QR_CUDA_TRY(launch_pdl(k_oz_sum, dim3((unsigned)ceil_div((long long)M * N, 256)), dim3(256), 0, st,
                           static_cast<const double2*>(w.part), splits, epi));
    note_launch();
    QR_CUDA_TRY(cudaGetLastError());
  }
  return QRTEBD_OK;
}

void tc_record_begin() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_recording = true;
  g_recorded.clear();
}

std::vector<TcShape> tc_record_end() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_recording = false;
  std::vector<TcShape> v;
  for (const TcShape& s : g_recorded) {
    bool seen = false;
    for (const TcShape& t : v) seen = seen || (!(s < t) && !(t < s));
    if (!seen) v.push_back(s);
  }
  g_recorded.clear();
  return v;
}

bool tc_tune_get(const TcShape& s, TcConfig* cfg) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(s);
  if (it == g_tune.end()) return false;
  *cfg = it->second.cfg;
  return true;
}

void tc_tune_put(const TcTuned& t) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[t.shape] = t;
}

std::vector<TcTuned> tc_tune_list() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  std::vector<TcTuned> v;
  for (const auto& kv : g_tune) v.push_back(kv.second);
  return v;
}

void tc_tune_clear() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune.clear();
}

int tc_tune_shape(const TcShape& s, cudaStream_t st, TcTuned* out) {
  // scratch operands of the shape (contiguous: the configurations differ only in the
  // tensor-core launches, which see the same prepared operands whatever the layout)
  const int M = s.M, N = s.N, K = s.K;
  if (M < N || N < 1 || K < 1) { set_last_message("autotune: bad shape"); return QRTEBD_ERR_INVALID_ARG; }
  ProfSuppress quiet;  // the candidates' launches are not part of any profiled work
  Arena ar;
  ar.measuring = true;
  TcWorkspace w;
  tc_carve(ar, M, K, N, w);
  const size_t ws_bytes = ar.off;
  const size_t na = (size_t)M * K, nb = (size_t)K * N, nc = (size_t)M * N;
  char* mem = nullptr;
  const size_t bytes = ws_bytes + 256 + (na + nb + nc) * sizeof(float2);
  QR_CUDA_TRY(cudaMalloc(&mem, bytes));
  int rc = QRTEBD_OK;
  do {
    Arena a2;
    a2.base = mem; a2.cap = ws_bytes;
    tc_carve(a2, M, K, N, w);
    float2* A = reinterpret_cast<float2*>(mem + align_up(ws_bytes, 256));
    float2* B = A + na;
    float2* C = B + nb;
    k_fill_test<<<(unsigned)ceil_div((long long)na, 256), 256, 0, st>>>(A, (long long)na, 1u);
    k_fill_test<<<(unsigned)ceil_div((long long)nb, 256), 256, 0, st>>>(B, (long long)nb, 2u);
    const float2 one = make_float2(1.f, 0.f), zero = make_float2(0.f, 0.f);
    GemmArgs<float> g{M, N, K, A, K, 1, false, B, N, 1, false, C, N, 1, one, zero};
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) { rc = QRTEBD_ERR_CUDA; break; }
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); rc = QRTEBD_ERR_CUDA; break; }
    auto time_cfg = [&](const TcConfig* c, double* ms) -> int {
      constexpr int kWarm = 2, kReps = 5;
      for (int i = 0; i < kWarm; ++i) QR_TRY(tc_gemm_cfg(g, s.three != 0, w, st, c));
      QR_CUDA_TRY(cudaEventRecord(e0, st));
      for (int i = 0; i < kReps; ++i) QR_TRY(tc_gemm_cfg(g, s.three != 0, w, st, c));
      QR_CUDA_TRY(cudaEventRecord(e1, st));
      QR_CUDA_TRY(cudaEventSynchronize(e1));
      float f = 0.f;
      QR_CUDA_TRY(cudaEventElapsedTime(&f, e0, e1));
      *ms = f / kReps;
      return QRTEBD_OK;
    };
    // the heuristic (no table entry consulted: an explicit default config)
    TcConfig heur;  // bn 256, heuristic splits, tail on
    double best_ms = 0.0, def_ms = 0.0;
    rc = time_cfg(&heur, &def_ms);
    if (rc != QRTEBD_OK) break;
    TcConfig best = heur;
    best_ms = def_ms;
    const int split_c[] = {1, 2, 3, 4, 6, 8, 12, 16, 24, 32};
    for (int bn : {256, 128}) {
      for (int sp : split_c) {
        for (int tail = 0; tail <= (sp == 1 ? 1 : 0); ++tail) {
          const int nx = (int)ceil_div(2LL * N, bn), ny = (int)ceil_div(M, BM);
          const int nk = (int)ceil_div(2LL * K, BK);
          if (sp > 1 && (sp > nk || (long long)nx * ny * sp > 8LL * 148 ||
                         (size_t)sp * M * 2 * N > w.p_cap))
            continue;
          TcConfig c{bn, sp, tail};
          double ms = 0.0;
          rc = time_cfg(&c, &ms);
          if (rc != QRTEBD_OK) break;
          if (ms < best_ms) { best_ms = ms; best = c; }
        }
        if (rc != QRTEBD_OK) break;
      }
      if (rc != QRTEBD_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != QRTEBD_OK) break;
    TcTuned t{s, best, best_ms, def_ms};
    tc_tune_put(t);
    if (out) *out = t;
  } while (false);
  cudaError_t fe = cudaStreamSynchronize(st);
  cudaFree(mem);
  if (rc == QRTEBD_OK && fe != cudaSuccess) { set_last_message(cudaGetErrorString(fe)); rc = QRTEBD_ERR_CUDA; }
  return rc;
}

}  // namespace qrtebd
