// Blocked Householder QR with explicit Q; see qr.cuh.
//
// Panel (nb columns): one thread-block cluster of up to 16 CTAs holds the panel
// in shared memory, each CTA a contiguous slab of rows. Every column needs two
// cluster-wide reductions - the reflector norm ||x||^2 (always FP64, with the
// pivot alpha riding along) and w = v^dag A_panel - done with partial sums in
// each CTA's shared memory, a hardware cluster barrier and distributed-shared-
// memory reads. Reflectors follow LAPACK's zlarfg convention
// (beta = -sign(Re alpha) ||(alpha, x)||, tau = (beta - alpha) / beta,
// v = [1, x / (alpha - beta)]), so R has a real diagonal. The panel also builds
// the compact-WY factor T (upper triangular, forward columnwise) from the Gram
// matrix V^dag V, so that H_1 ... H_nb = I - V T V^dag.
//
// Trailing update per panel:   C <- (I - V T V^dag)^dag C = C - V (T^dag (V^dag C))
// Explicit Q (backward):       Q[k0:, k0:] <- (I - V T V^dag) Q[k0:, k0:], Q = [I; 0] initially
// The three contractions of each step go through QrGemm (CUDA cores by default,
// tcgen05 tensor cores in the complex64 tensor-core path).
#include <cooperative_groups.h>

#include <limits>
#include <map>
#include <mutex>
#include <vector>

#include "qr.cuh"

namespace cg = cooperative_groups;

namespace qrtebd {

namespace {

constexpr int PT = 256;      // threads per panel CTA
constexpr int KBMAX = 32;    // widest panel
constexpr int NBO = 128;     // outer block of the two-level blocking
constexpr int RED = 3 * 16 + 4;  // 3 doubles per cluster rank
constexpr int SMEM_CAP = 220 * 1024;

template <typename T> struct PanelArgs {
  cx<T>* A; long long lda; int m; int k0; int kb;
  cx<T>* V; long long ldv;
  cx<T>* tau; cx<T>* Tf; int ldt;
  int rpc; unsigned* err;
};

__host__ __device__ inline size_t a16(size_t x) { return (x + 15) & ~size_t(15); }

template <typename T> struct PanelSmem;
template <typename T> __host__ __device__ inline size_t panel_smem_bytes(int rpc, int kb);

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <typename T> __device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------- panel kernel
// One 32-column Householder panel on a cluster of CS CTAs; CTA r holds panel rows
// [r*rpc, (r+1)*rpc) in shared memory. Per column j:
//   A. partial ||x||^2 below the pivot and alpha, summed over the CTA's warps;
//   B. all-to-all: every CTA copies its partial into slot [rank] of every CTA's
//      receive buffer with one cp.async.bulk (distributed shared memory) whose
//      completion is counted on the receiver's mbarrier; no cluster barrier;
//   C. every thread forms the reflector (zlarfg convention) from the CS partials;
//   D. per-warp rows: v = x * scale, dot products with lane = slot: slots < nc give
//      w_c = v^dag P[:, c], slots >= nc give g_a = v_a^dag v (compact-WY T column);
//   E. all-to-all of the slot partials as in B;
//   F. P[:, c] -= v conj(tau) w_c (lane = column), T(0:j, j) = -tau T(0:j, 0:j) g.
// The norm accumulates in double-float for complex64 (two FP32 words, error-free
// FMA products and TwoSum additions, ~48-bit significand) and in FP64 for complex128:
// B300's FP64 pipe is too narrow for the panel's critical path, and the reflector is
// stored in FP32 anyway, so FP64-class accuracy is what the norm needs.
template <typename T> struct NAcc;  // norm accumulator: double-float (float) or FP64 (double)
template <> struct NAcc<float> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float a, float b) {  // += (a_hi, a_lo) pair
    const float s = hi + a, bb = s - hi, e = (hi - (s - bb)) + (a - bb);
    const float t = e + lo + b;
    hi = s + t; lo = t - (hi - s);
  }
  __device__ __forceinline__ void add_sq(float x) { const float p = x * x; add(p, fmaf(x, x, -p)); }
  __device__ __forceinline__ void add(const NAcc& o) { add(o.hi, o.lo); }
  __device__ __forceinline__ void shfl_sum() {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float h = __shfl_xor_sync(0xffffffffu, hi, o), l = __shfl_xor_sync(0xffffffffu, lo, o);
      add(h, l);
    }
  }
  __device__ __forceinline__ float value() const { return hi + lo; }
};
template <> struct NAcc<double> {
  double v = 0.0;
  __device__ __forceinline__ void add(double a, double b) { v += a + b; }
  __device__ __forceinline__ void add_sq(double x) { v = fma(x, x, v); }
  __device__ __forceinline__ void add(const NAcc& o) { v += o.v; }
  __device__ __forceinline__ void shfl_sum() {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  }
  __device__ __forceinline__ double value() const { return v; }
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint32_t map_rank(uint32_t a, int rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ void mbar_init1(uint64_t* b) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(b)) : "memory");
}
__device__ __forceinline__ void mbar_arm(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)),
               "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_wait_cl(uint64_t* b, uint32_t parity) {
  for (long long i = 0; i < kSpinLimit; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok) : "r"(smem_addr(b)), "r"(parity) : "memory");
    if (ok) return true;
  }
  return false;
}
// copy `bytes` (multiple of 16) from this CTA's shared memory to CTA `rank`, counted on
// that CTA's mbarrier
__device__ __forceinline__ void dsmem_send(const void* src, void* dst_local, uint64_t* mbar_local,
                                           int rank, uint32_t bytes) {
  const uint32_t d = map_rank(smem_addr(dst_local), rank);
  const uint32_t m = map_rank(smem_addr(mbar_local), rank);
  asm volatile(
      "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(d), "r"(smem_addr(src)), "r"(bytes), "r"(m) : "memory");
}

constexpr int SLOTS = KBMAX;              // slot partials per exchange (padded)

template <typename T> struct PanelSmem {
  // per-column exchange buffers, double-buffered by column parity
  static constexpr int R1 = 4;            // reduction-1 payload: norm (hi, lo) or (v, 0), alpha re, im
  static constexpr size_t fixed() {
    return a16(2 * 16 * R1 * sizeof(T))            // recv1 [2][16][R1]
         + a16(R1 * sizeof(T))                     // send1
         + a16(2 * 16 * SLOTS * sizeof(cx<T>))     // recv2 [2][16][SLOTS]
         + a16(SLOTS * sizeof(cx<T>))              // send2
         + a16(8 * R1 * sizeof(T))                 // per-warp reduction-1 partials
         + a16(8 * SLOTS * sizeof(cx<T>))          // per-warp slot partials
         + a16(KBMAX * sizeof(cx<T>))              // taus
         + a16(KBMAX * (KBMAX + 1) * sizeof(cx<T>))  // T
         + 64;                                     // 4 mbarriers
  }
};

template <typename T> __host__ __device__ inline size_t panel_smem_bytes(int rpc, int kb) {
  return a16((size_t)rpc * (kb + 1) * sizeof(cx<T>)) + a16((size_t)rpc * sizeof(cx<T>)) +
         PanelSmem<T>::fixed();
}

template <typename T>
__global__ void __launch_bounds__(PT) k_qr_panel(PanelArgs<T> a) {
  extern __shared__ __align__(16) unsigned char sm[];
  cg::cluster_group cl = cg::this_cluster();
  const int CS = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = PT / 32;
  constexpr int R1 = PanelSmem<T>::R1;
  const int kb = a.kb, ldp = kb + 1, rpc = a.rpc;
  const int mr = a.m - a.k0;
  const int row0 = rank * rpc;
  const int nloc = max(0, min(rpc, mr - row0));
  const int rpw = (nloc + NW - 1) / NW;              // rows per warp
  const int p0 = min(nloc, warp * rpw), p1 = min(nloc, p0 + rpw);

  unsigned char* q = sm;
  cx<T>* P = reinterpret_cast<cx<T>*>(q); q += a16((size_t)rpc * ldp * sizeof(cx<T>));
  cx<T>* VV = reinterpret_cast<cx<T>*>(q); q += a16((size_t)rpc * sizeof(cx<T>));
  T* recv1 = reinterpret_cast<T*>(q); q += a16(2 * 16 * R1 * sizeof(T));
  T* send1 = reinterpret_cast<T*>(q); q += a16(R1 * sizeof(T));
  cx<T>* recv2 = reinterpret_cast<cx<T>*>(q); q += a16(2 * 16 * SLOTS * sizeof(cx<T>));
  cx<T>* send2 = reinterpret_cast<cx<T>*>(q); q += a16(SLOTS * sizeof(cx<T>));
  T* wp1 = reinterpret_cast<T*>(q); q += a16(8 * R1 * sizeof(T));
  cx<T>* wp2 = reinterpret_cast<cx<T>*>(q); q += a16(8 * SLOTS * sizeof(cx<T>));
  cx<T>* taus = reinterpret_cast<cx<T>*>(q); q += a16(KBMAX * sizeof(cx<T>));
  cx<T>* Ts = reinterpret_cast<cx<T>*>(q); q += a16(KBMAX * (KBMAX + 1) * sizeof(cx<T>));
  uint64_t* mb = reinterpret_cast<uint64_t*>(q);     // mb[0..1] reduction 1, mb[2..3] reduction 2

  const long long k0 = a.k0;
  for (int idx = tid; idx < nloc * kb; idx += PT) {
    const int p = idx / kb, c = idx % kb;
    P[p * ldp + c] = a.A[(k0 + row0 + p) * a.lda + k0 + c];
  }
  if (tid == 0) {
    for (int i = 0; i < 4; ++i) mbar_init1(&mb[i]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  cl.sync();  // every CTA's barriers exist before anyone sends
  bool ok = true;

  for (int j = 0; j < kb; ++j) {
    const int buf = j & 1;
    const uint32_t ph = (uint32_t)((j >> 1) & 1);
    // ---- A: partial norm below the pivot, alpha
    {
      NAcc<T> acc;
      T ar = 0, ai = 0;
      for (int p = p0 + lane; p < p1; p += 32) {
        const int g = row0 + p;
        const cx<T> v = P[p * ldp + j];
        if (g > j) { acc.add_sq(v.x); acc.add_sq(v.y); }
        else if (g == j) { ar = v.x; ai = v.y; }
      }
      acc.shfl_sum();
      ar = warp_sum_t<T>(ar); ai = warp_sum_t<T>(ai);
      if (lane == 0) {
        if constexpr (std::is_same<T, float>::value) { wp1[warp * R1 + 0] = acc.hi; wp1[warp * R1 + 1] = acc.lo; }
        else { wp1[warp * R1 + 0] = acc.value(); wp1[warp * R1 + 1] = 0; }
        wp1[warp * R1 + 2] = ar; wp1[warp * R1 + 3] = ai;
      }
    }
    __syncthreads();
    if (warp == 0) {
      if (lane == 0) {
        NAcc<T> s;
        T ar = 0, ai = 0;
        for (int w = 0; w < NW; ++w) { s.add(wp1[w * R1], wp1[w * R1 + 1]); ar += wp1[w * R1 + 2]; ai += wp1[w * R1 + 3]; }
        if constexpr (std::is_same<T, float>::value) { send1[0] = s.hi; send1[1] = s.lo; }
        else { send1[0] = s.value(); send1[1] = 0; }
        send1[2] = ar; send1[3] = ai;
        mbar_arm(&mb[buf], (uint32_t)(CS * R1 * sizeof(T)));
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      }
      __syncwarp();
      if (lane < CS)
        dsmem_send(send1, recv1 + (buf * 16 + rank) * R1, &mb[buf], lane, R1 * sizeof(T));
    }
    if (!mbar_wait_cl(&mb[buf], ph)) ok = false;
    // ---- C: the reflector, redundantly in every thread (working precision only)
    T beta, tr, ti, sr, si;
    {
      // every warp sums the CS partials with a shuffle tree (lane r holds rank r's)
      NAcc<T> s;
      T alr = 0, ali = 0;
      if (lane < CS) {
        const T* rr = recv1 + (buf * 16 + lane) * R1;
        s.add(rr[0], rr[1]); alr = rr[2]; ali = rr[3];
      }
      s.shfl_sum();
      alr = warp_sum_t<T>(alr); ali = warp_sum_t<T>(ali);
      const T xn2 = s.value();
      beta = alr; tr = ti = sr = si = T(0);
      // A column whose squared norm is below the normal range (noise of a rank-deficient
      // block) is left as is: tau = 0, H = I, which is exactly unitary.
      const T tot = alr * alr + ali * ali + xn2;
      if (!(xn2 == T(0) && ali == T(0)) && tot > T(16) * std::numeric_limits<T>::min()) {
        const T nrm = sqrt(tot);
        beta = alr >= T(0) ? -nrm : nrm;
        tr = (beta - alr) / beta;
        ti = -ali / beta;
        const T dr = alr - beta, di = ali;  // scale = 1 / (alpha - beta), Smith's division
        if (fabs(dr) >= fabs(di)) { const T rt = di / dr, den = dr + di * rt; sr = T(1) / den; si = -rt / den; }
        else { const T rt = dr / di, den = di + dr * rt; sr = rt / den; si = T(-1) / den; }
      }
      if (tid == 0 && rank == 0 && !(isfinite(beta) && isfinite(sr) && isfinite(si)))
        atomicOr(a.err, DEVERR_NUMERIC);
    }
    const cx<T> scale = mk<T>(sr, si), tau = mk<T>(tr, ti);
    if (tid == 0) taus[j] = tau;
    // ---- D: v for this warp's rows, then slot partials (lane = slot)
    const int nc = kb - j - 1;
    const int nslot = nc + j;
    for (int p = p0 + lane; p < p1; p += 32) {
      const int g = row0 + p;
      if (g > j) VV[p] = cmul<T>(P[p * ldp + j], scale);
      else if (g == j) VV[p] = mk<T>(1, 0);
    }
    __syncwarp();
    if (nslot > 0) {
      cx<T> acc = mk<T>(0, 0);
      if (lane < nslot) {
        // slot < nc: conj(v) . P[:, c];  slot >= nc: conj(v_a) . v  (= conj of v^dag v_a)
        const bool is_w = lane < nc;
        const int col = is_w ? j + 1 + lane : lane - nc;
        const T sg = is_w ? T(1) : T(-1);
        cx<T> a0 = mk<T>(0, 0), a1 = mk<T>(0, 0), a2 = mk<T>(0, 0), a3 = mk<T>(0, 0);
        int p = max(p0, j - row0);
        for (; p + 3 < p1; p += 4) {
          cx<T> v, x;
          v = VV[p]; x = P[p * ldp + col];
          a0.x += v.x * x.x + v.y * x.y; a0.y += v.x * x.y - v.y * x.x;
          v = VV[p + 1]; x = P[(p + 1) * ldp + col];
          a1.x += v.x * x.x + v.y * x.y; a1.y += v.x * x.y - v.y * x.x;
          v = VV[p + 2]; x = P[(p + 2) * ldp + col];
          a2.x += v.x * x.x + v.y * x.y; a2.y += v.x * x.y - v.y * x.x;
          v = VV[p + 3]; x = P[(p + 3) * ldp + col];
          a3.x += v.x * x.x + v.y * x.y; a3.y += v.x * x.y - v.y * x.x;
        }
        for (; p < p1; ++p) {
          const cx<T> v = VV[p], x = P[p * ldp + col];
          a0.x += v.x * x.x + v.y * x.y; a0.y += v.x * x.y - v.y * x.x;
        }
        acc.x = (a0.x + a1.x) + (a2.x + a3.x);
        acc.y = sg * ((a0.y + a1.y) + (a2.y + a3.y));
      }
      wp2[warp * SLOTS + lane] = acc;
      __syncthreads();
      if (warp == 0) {
        cx<T> s = mk<T>(0, 0);
        for (int w = 0; w < NW; ++w) s = cadd<T>(s, wp2[w * SLOTS + lane]);
        send2[lane] = s;
        // every sender copies its nslot values rounded up to 16 bytes
        const uint32_t bytes = (uint32_t)(nslot * sizeof(cx<T>) + 15) & ~15u;
        if (lane == 0) mbar_arm(&mb[2 + buf], (uint32_t)CS * bytes);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane < CS) dsmem_send(send2, recv2 + (buf * 16 + rank) * SLOTS, &mb[2 + buf], lane, bytes);
      }
      if (!mbar_wait_cl(&mb[2 + buf], ph)) ok = false;
      // ---- F: update (lane = column) and the T column
      cx<T> w = mk<T>(0, 0);
      if (lane < nslot) {
        const cx<T>* rr = recv2 + buf * 16 * SLOTS + lane;
        for (int r = 0; r < CS; ++r) w = cadd<T>(w, rr[r * SLOTS]);
      }
      if (lane < nc) {
        const cx<T> cw = cmul<T>(cconj<T>(tau), w);  // conj(tau) w_c
        cx<T>* col = P + j + 1 + lane;
        int p = max(p0, j - row0);
        for (; p + 1 < p1; p += 2) {
          const cx<T> x0 = col[p * ldp], x1 = col[(p + 1) * ldp];
          const cx<T> v0 = VV[p], v1 = VV[p + 1];
          col[p * ldp] = csub<T>(x0, cmul<T>(v0, cw));
          col[(p + 1) * ldp] = csub<T>(x1, cmul<T>(v1, cw));
        }
        if (p < p1) col[p * ldp] = csub<T>(col[p * ldp], cmul<T>(VV[p], cw));
      }
      // g_a = v_a^dag v_j (a < j) is kept in column j of Ts for the T recurrence at the end
      if (warp == 0 && lane >= nc && lane < nslot) Ts[(lane - nc) * (KBMAX + 1) + j] = w;
    }
    // column j <- v below the pivot, beta on it
    for (int p = p0 + lane; p < p1; p += 32) {
      const int g = row0 + p;
      if (g > j) P[p * ldp + j] = VV[p];
      else if (g == j) P[p * ldp + j] = mk<T>(beta, T(0));
    }
    __syncthreads();
  }
  if (!ok && tid == 0) atomicOr(a.err, DEVERR_TIMEOUT);

  // compact-WY T, column by column (forward, columnwise): Ts[0:j, j] holds g = V^dag v_j,
  // T(0:j, j) = -tau_j T(0:j, 0:j) g, T(j, j) = tau_j
  if (rank == 0 && warp == 0) {
    for (int j = 0; j < kb; ++j) {
      const cx<T> tj = taus[j];
      cx<T> acc2 = mk<T>(0, 0);
      if (lane < j)
        for (int l = lane; l < j; ++l) cfma<T>(acc2, Ts[lane * (KBMAX + 1) + l], Ts[l * (KBMAX + 1) + j]);
      __syncwarp();
      if (lane < j) { const cx<T> r = cmul<T>(tj, acc2); Ts[lane * (KBMAX + 1) + j] = mk<T>(-r.x, -r.y); }
      if (lane == j) Ts[j * (KBMAX + 1) + j] = tj;
      __syncwarp();
    }
  }
  __syncthreads();

  if (rank == 0) {
    for (int idx = tid; idx < kb * kb; idx += PT) {
      const int i = idx / kb, jj = idx % kb;
      a.Tf[i * a.ldt + jj] = (jj >= i) ? Ts[i * (KBMAX + 1) + jj] : mk<T>(0, 0);
    }
    if (tid < kb) a.tau[k0 + tid] = taus[tid];
  }
  // ---- write V (explicit, unit lower trapezoidal) and R / zeros into A
  for (int idx = tid; idx < nloc * kb; idx += PT) {
    const int p = idx / kb, c = idx % kb;
    const int g = row0 + p;
    const cx<T> pv = P[p * ldp + c];
    a.V[(k0 + g) * a.ldv + k0 + c] = (g == c) ? mk<T>(1, 0) : (g > c ? pv : mk<T>(0, 0));
    a.A[(k0 + g) * a.lda + k0 + c] = (c >= g) ? pv : mk<T>(0, 0);
  }
  cl.sync();  // no CTA exits while a copy into its shared memory could be pending
}

template <typename T>
__global__ void k_eye(cx<T>* Q, long long ldq, int m, int n) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)m * n) return;
  int i = (int)(idx / n), j = (int)(idx % n);
  Q[i * ldq + j] = mk<T>(i == j ? T(1) : T(0), 0);
}

struct ClusterChoice { int cs; int rpc; int kb; };

// Largest cluster the device co-schedules for the panel kernel (16 needs the
// non-portable opt-in; probed once per process, falls back to 8).
int g_max_cluster = 0;

template <typename T> ClusterChoice choose_cluster(int mr, int kb_want) {
  ClusterChoice c{1, mr, kb_want};
  const int cmax = g_max_cluster > 0 ? g_max_cluster : 16;
  int cs = 1;
  while (cs < cmax && (long long)cs * 192 < mr) cs *= 2;
  for (int kb = kb_want; kb >= 1; kb /= 2) {
    for (int s = cs; s <= cmax; s *= 2) {
      int rpc = (int)ceil_div(mr, s);
      if (panel_smem_bytes<T>(rpc, kb) <= (size_t)SMEM_CAP) return ClusterChoice{s, rpc, kb};
    }
  }
  c.cs = -1;
  return c;
}

template <typename T> bool g_attr_done = false;

// Probe once whether 16-CTA clusters of the panel kernel (at the largest shared
// memory size) can be co-scheduled; otherwise cap clusters at 8 CTAs.
template <typename T> int probe_max_cluster() {
  if (g_max_cluster > 0) return QRTEBD_OK;
  QR_CUDA_TRY(cudaFuncSetAttribute(k_qr_panel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_CAP));
  QR_CUDA_TRY(cudaFuncSetAttribute(k_qr_panel<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  g_attr_done<T> = true;
  cudaLaunchConfig_t q = {};
  q.gridDim = dim3(16, 1, 1); q.blockDim = dim3(PT, 1, 1); q.dynamicSmemBytes = SMEM_CAP;
  cudaLaunchAttribute qa[1];
  qa[0].id = cudaLaunchAttributeClusterDimension;
  qa[0].val.clusterDim.x = 16; qa[0].val.clusterDim.y = 1; qa[0].val.clusterDim.z = 1;
  q.attrs = qa; q.numAttrs = 1;
  int nclusters = 0;
  cudaError_t e = cudaOccupancyMaxActiveClusters(&nclusters, k_qr_panel<T>, &q);
  if (e != cudaSuccess) (void)cudaGetLastError();
  g_max_cluster = (e == cudaSuccess && nclusters >= 1) ? 16 : 8;
  return QRTEBD_OK;
}

template <typename T> int launch_panel(const PanelArgs<T>& pa, int cs, cudaStream_t st) {
  size_t smem = panel_smem_bytes<T>(pa.rpc, pa.kb);
  if (!g_attr_done<T>) {
    QR_CUDA_TRY(cudaFuncSetAttribute(k_qr_panel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_CAP));
    QR_CUDA_TRY(cudaFuncSetAttribute(k_qr_panel<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    g_attr_done<T> = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cs, 1, 1);
  cfg.blockDim = dim3(PT, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs; attr[0].val.clusterDim.y = 1; attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr; cfg.numAttrs = 1;
  ProfScope prof(PROF_QR_PANEL, st);
  QR_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_qr_panel<T>, pa));
  note_launch();
  return QRTEBD_OK;
}

// Side streams for look-ahead, one per (device, main stream), with reusable events.
struct SideStream {
  cudaStream_t st = nullptr;
  std::vector<cudaEvent_t> ev;
};
std::mutex g_side_mu;
std::map<std::pair<int, cudaStream_t>, SideStream> g_side;

int side_stream(cudaStream_t main, int nev, SideStream** out) {
  int dev = 0;
  QR_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_side_mu);
  SideStream& ss = g_side[std::make_pair(dev, main)];
  if (!ss.st) QR_CUDA_TRY(cudaStreamCreateWithFlags(&ss.st, cudaStreamNonBlocking));
  while ((int)ss.ev.size() < nev) {
    cudaEvent_t e;
    QR_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    ss.ev.push_back(e);
  }
  *out = &ss;
  return QRTEBD_OK;
}

template <typename T>
int run_gemm(const GemmArgs<T>& g, const QrScratch<T>& s, cudaStream_t st, const QrGemm<T>* gm) {
  if (gm && gm->fn) return gm->fn(g, st, gm->ctx);
  return gemm_simt<T>(g, st, s.gemm_scratch, s.gemm_scratch_elems);
}

}  // namespace

int qr_panel_width(int m, int n, int elem_bytes) {
  int kb = n < KBMAX ? n : KBMAX;
  if (kb < 1) kb = 1;
  if (elem_bytes == 16) {
    ClusterChoice c = choose_cluster<double>(m, kb);
    return c.cs < 0 ? -1 : c.kb;
  }
  ClusterChoice c = choose_cluster<float>(m, kb);
  return c.cs < 0 ? -1 : c.kb;
}

template <typename T> void qr_carve(Arena& ar, int m, int n, QrScratch<T>& s) {
  // one NBO x NBO compact-WY factor per outer block; W, W2 hold NBO x n
  const int nbo = NBO;
  s.V = ar.take<cx<T>>((size_t)m * n);
  s.tau = ar.take<cx<T>>(n);
  s.Tf = ar.take<cx<T>>((size_t)(n + nbo) * nbo);
  s.W = ar.take<cx<T>>((size_t)nbo * n);
  s.W2 = ar.take<cx<T>>((size_t)nbo * n);
  s.Ws = ar.take<cx<T>>((size_t)nbo * n);
  s.W2s = ar.take<cx<T>>((size_t)nbo * n);
  s.G = ar.take<cx<T>>((size_t)nbo * nbo);
  s.tmp = ar.take<cx<T>>((size_t)nbo * KBMAX);
  size_t e = 0;
  for (int k = 1; k <= nbo; k *= 2) {
    e = std::max(e, gemm_simt_scratch_elems(k, n, m, 1));
    e = std::max(e, gemm_simt_scratch_elems(k, k, m, 1));
  }
  e = std::max(e, gemm_simt_scratch_elems(m, n, nbo, 1));
  s.gemm_scratch_elems = e;
  s.gemm_scratch = e ? ar.take<cx<T>>(e) : nullptr;
}

template <typename T>
int householder_qr(cx<T>* A, long long lda, int m, int n, cx<T>* Q, long long ldq,
                   QrScratch<T>& s, cudaStream_t st, unsigned* err, const QrGemm<T>* gm,
                   const QrGemm<T>* side) {
  if (m < n || n < 1) return QRTEBD_ERR_INVALID_ARG;
  QR_TRY(probe_max_cluster<T>());
  const int nb = qr_panel_width(m, n, sizeof(cx<T>));
  if (nb < 1) { set_last_message("QR: matrix too tall for the shared-memory panel"); return QRTEBD_ERR_INVALID_ARG; }
  const long long ldv = n;
  const int nbo = NBO;  // outer block: inner panels of nb columns inside it
  const cx<T> one = mk<T>(1, 0), zero = mk<T>(0, 0), mone = mk<T>(-1, 0);
  // V must be zero above each panel's diagonal block: an outer block reads the rows
  // above its later inner panels, which those panels do not write
  QR_CUDA_TRY(cudaMemsetAsync(s.V, 0, (size_t)m * n * sizeof(cx<T>), st));

  const int nblk = (int)ceil_div(n, nbo);
  SideStream* ss = nullptr;
  if (side && side->fn && nblk > 2) QR_TRY(side_stream(st, 2 * nblk, &ss));
  std::vector<char> rec(nblk, 0);  // which blocks recorded a side-stream update
  // latest side-stream update of a block <= k (the side stream runs them in order)
  auto latest = [&](int k) { for (int j = std::min(k, nblk - 1); j >= 0; --j) if (rec[j]) return j; return -1; };
  for (int ko = 0; ko < n; ko += nbo) {
    const int kbo = std::min(nbo, n - ko);
    const int mo = m - ko;
    const int kblk = ko / nbo;
    // this block's columns must have received the side-stream updates of blocks <= k-2
    if (ss && latest(kblk - 2) >= 0)
      QR_CUDA_TRY(cudaStreamWaitEvent(st, ss->ev[nblk + latest(kblk - 2)], 0));
    cx<T>* Tb = s.Tf + (size_t)(ko / nbo) * nbo * nbo;
    QR_CUDA_TRY(cudaMemsetAsync(Tb, 0, (size_t)nbo * nbo * sizeof(cx<T>), st));
    for (int ki = ko; ki < ko + kbo; ki += nb) {
      const int kb = std::min(nb, ko + kbo - ki);
      const int mr = m - ki;
      ClusterChoice cc = choose_cluster<T>(mr, kb);
      if (cc.cs < 0 || cc.kb != kb) { cc.kb = kb; cc.cs = 16; cc.rpc = (int)ceil_div(mr, 16); }
      cx<T>* Ti = Tb + (size_t)(ki - ko) * nbo + (ki - ko);
      PanelArgs<T> pa{A, lda, m, ki, kb, s.V, ldv, s.tau, Ti, nbo, cc.rpc, err};
      QR_TRY(launch_panel<T>(pa, cc.cs, st));
      // inner update: the rest of this outer block
      const int nc = ko + kbo - ki - kb;
      if (nc > 0) {
        const cx<T>* Vk = s.V + (long long)ki * ldv + ki;
        cx<T>* C = A + (long long)ki * lda + ki + kb;
        GemmArgs<T> g1{kb, nc, mr, Vk, 1, ldv, true, C, lda, 1, false, s.W, nc, 1, one, zero};
        QR_TRY(gemm_simt<T>(g1, st, s.gemm_scratch, s.gemm_scratch_elems));
        GemmArgs<T> g2{kb, nc, kb, Ti, 1, nbo, true, s.W, nc, 1, false, s.W2, nc, 1, one, zero};
        QR_TRY(gemm_simt<T>(g2, st, s.gemm_scratch, s.gemm_scratch_elems));
        GemmArgs<T> g3{mr, nc, kb, Vk, ldv, 1, false, s.W2, nc, 1, false, C, lda, 1, mone, one};
        QR_TRY(run_gemm<T>(g3, s, st, gm));
      }
    }
    const cx<T>* Vb = s.V + (long long)ko * ldv + ko;
    if (kbo > nb) {
      // T of the outer block from the inner ones: with G = V^dag V,
      // T[0:c0, c0:c0+w] = -T[0:c0, 0:c0] G[0:c0, c0:c0+w] T[c0:c0+w, c0:c0+w]
      GemmArgs<T> gg{kbo, kbo, mo, Vb, 1, ldv, true, Vb, ldv, 1, false, s.G, nbo, 1, one, zero};
      QR_TRY(run_gemm<T>(gg, s, st, gm));
      for (int c0 = nb; c0 < kbo; c0 += nb) {
        const int w = std::min(nb, kbo - c0);
        GemmArgs<T> t1{c0, w, w, s.G + c0, nbo, 1, false, Tb + (size_t)c0 * nbo + c0, nbo, 1, false,
                       s.tmp, w, 1, one, zero};
        QR_TRY(gemm_simt<T>(t1, st, s.gemm_scratch, s.gemm_scratch_elems));
        GemmArgs<T> t2{c0, w, c0, Tb, nbo, 1, false, s.tmp, w, 1, false, Tb + c0, nbo, 1, mone, zero};
        QR_TRY(gemm_simt<T>(t2, st, s.gemm_scratch, s.gemm_scratch_elems));
      }
    }
    // outer trailing update: C <- (I - V T V^dag)^dag C. With look-ahead the next outer
    // block's columns are updated here and the rest on the side stream, overlapping the
    // next block's panels.
    const int nc = n - ko - kbo;
    if (nc > 0) {
      auto update = [&](int c0, int cw, cudaStream_t stream, cx<T>* W, cx<T>* W2,
                        const QrGemm<T>* g) -> int {
        cx<T>* C = A + (long long)ko * lda + ko + kbo + c0;
        GemmArgs<T> g1{kbo, cw, mo, Vb, 1, ldv, true, C, lda, 1, false, W, cw, 1, one, zero};
        QR_TRY(run_gemm<T>(g1, s, stream, g));
        GemmArgs<T> g2{kbo, cw, kbo, Tb, 1, nbo, true, W, cw, 1, false, W2, cw, 1, one, zero};
        QR_TRY(run_gemm<T>(g2, s, stream, g));
        GemmArgs<T> g3{mo, cw, kbo, Vb, ldv, 1, false, W2, cw, 1, false, C, lda, 1, mone, one};
        QR_TRY(run_gemm<T>(g3, s, stream, g));
        return QRTEBD_OK;
      };
      const int n1 = ss ? std::min(nbo, nc) : nc;
      // the next block's columns also carry block k-1's side-stream update: order after it
      if (ss && latest(kblk - 1) >= 0)
        QR_CUDA_TRY(cudaStreamWaitEvent(st, ss->ev[nblk + latest(kblk - 1)], 0));
      QR_TRY(update(0, n1, st, s.W, s.W2, gm));
      if (ss && nc > n1) {
        QR_CUDA_TRY(cudaEventRecord(ss->ev[kblk], st));  // V, T of this block are ready
        QR_CUDA_TRY(cudaStreamWaitEvent(ss->st, ss->ev[kblk], 0));
        QR_TRY(update(n1, nc - n1, ss->st, s.Ws, s.W2s, side));
        QR_CUDA_TRY(cudaEventRecord(ss->ev[nblk + kblk], ss->st));
        rec[kblk] = 1;
      }
    }
  }
  if (ss && latest(nblk - 1) >= 0)
    QR_CUDA_TRY(cudaStreamWaitEvent(st, ss->ev[nblk + latest(nblk - 1)], 0));

  // explicit Q by backward accumulation over the outer blocks
  {
    long long tot = (long long)m * n;
    k_eye<T><<<(unsigned)ceil_div(tot, 256), 256, 0, st>>>(Q, ldq, m, n);
    note_launch();
    QR_CUDA_TRY(cudaGetLastError());
  }
  const int npo = (int)ceil_div(n, nbo);
  for (int p = npo - 1; p >= 0; --p) {
    const int ko = p * nbo;
    const int kbo = std::min(nbo, n - ko);
    const int mo = m - ko, nq = n - ko;
    const cx<T>* Vb = s.V + (long long)ko * ldv + ko;
    const cx<T>* Tb = s.Tf + (size_t)p * nbo * nbo;
    cx<T>* Qs = Q + (long long)ko * ldq + ko;
    GemmArgs<T> g1{kbo, nq, mo, Vb, 1, ldv, true, Qs, ldq, 1, false, s.W, nq, 1, one, zero};
    QR_TRY(run_gemm<T>(g1, s, st, gm));
    GemmArgs<T> g2{kbo, nq, kbo, Tb, nbo, 1, false, s.W, nq, 1, false, s.W2, nq, 1, one, zero};
    QR_TRY(run_gemm<T>(g2, s, st, gm));
    GemmArgs<T> g3{mo, nq, kbo, Vb, ldv, 1, false, s.W2, nq, 1, false, Qs, ldq, 1, mone, one};
    QR_TRY(run_gemm<T>(g3, s, st, gm));
  }
  return QRTEBD_OK;
}

template void qr_carve<float>(Arena&, int, int, QrScratch<float>&);
template void qr_carve<double>(Arena&, int, int, QrScratch<double>&);
template int householder_qr<float>(float2*, long long, int, int, float2*, long long,
                                   QrScratch<float>&, cudaStream_t, unsigned*, const QrGemm<float>*,
                                   const QrGemm<float>*);
template int householder_qr<double>(double2*, long long, int, int, double2*, long long,
                                    QrScratch<double>&, cudaStream_t, unsigned*,
                                    const QrGemm<double>*, const QrGemm<double>*);

}  // namespace qrtebd
