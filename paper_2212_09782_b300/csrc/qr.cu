// Blocked Householder QR with explicit Q; see qr.cuh.
//
// Panel (nb columns): one thread-block cluster of up to 16 CTAs holds the panel
// in shared memory: every CTA a copy of the panel's first nb rows (the pivot rows)
// and a contiguous slab of the rows below. Every column needs one cluster-wide
// reduction - the reflector norm together with the raw column dot products, from
// which w = v^dag A_panel follows - pushed into every CTA's shared memory by remote
// stores that complete on the receiver's mbarrier. Reflectors follow LAPACK's zlarfg
// convention (beta = -sign(Re alpha) ||(alpha, x)||, tau = (beta - alpha) / beta,
// v = [1, x / (alpha - beta)]), so R has a real diagonal. The panel also builds the
// compact-WY factor T (upper triangular) from the Gram values v_a^dag v_j, so that
// H_1 ... H_nb = I - V T V^dag.
//
// Trailing update per block:   C <- (I - V T V^dag)^dag C = C - V ((V T)^dag C)
// Explicit Q (backward):       Q[k0:, k0:] <- Q[k0:, k0:] - (V T)(V^dag Q[k0:, k0:]), Q = [I; 0]
// with V T formed once per outer block.
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
constexpr int PG_MAX = 148;  // CTAs of the complex128 grid panel (one per SM at most)

template <typename T> struct PanelArgs {
  cx<T>* A; long long lda; int m; int k0; int kb;
  cx<T>* V; long long ldv;
  cx<T>* tau; cx<T>* Tf; int ldt;
  int rps; unsigned* err;  // rps: slab rows per CTA below the replicated first kb rows
};

__host__ __device__ inline size_t a16(size_t x) { return (x + 15) & ~size_t(15); }


template <typename T> __device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------- panel kernel
// One Householder panel of kb <= 32 columns on a cluster of CS CTAs. Local rows of
// every CTA: the panel's first kb rows (a replica, updated identically everywhere, so
// each CTA has the pivot row of every column) followed by its slab of rps rows below;
// the replica enters rank 0's partial sums only.
// A reflector needs ||x||^2 below its pivot and w_c = v^dag P[:, c] for the columns it
// updates. With v = scale * x below the pivot and 1 on it, w_c = P[j, c] + conj(scale) S_c
// where S_c = sum_{g > j} conj(x_g) P[g, c] does not depend on scale; the Gram values of
// the compact-WY factor, g_a = v_a^dag v_j, come from the same sums. So each column takes
// ONE cluster-wide exchange of (||x||^2 partial, S_c partials), and the pass over the rows
// that applies reflector j also forms the partials of column j+1:
//   1. lane = row: v of reflector j, column j+1 updated in place, ||x_{j+1}||^2 partial;
//   2. lane = column c: P[:, c] -= v conj(tau) w_c (c > j+1), S_c partial (every c);
//   3. warp 0 sums the warps' partials and pushes them to every CTA: 16-byte st.async
//      remote stores, counted on the receiver's mbarrier (double-buffered by parity);
//   4. warp 0 forms the next reflector (zlarfg convention) and conj(tau) w_c for every
//      column, and hands them to the other warps through shared memory.
// Columns are stored raw (x, not v) during the panel; v = scale * x is written at the
// end. T comes last, by recursive doubling over the Gram values.
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
  // the pair = x^2 + y^2 (error-free products, TwoSum of their high words)
  __device__ __forceinline__ void set_abs2(float x, float y) {
    const float a = x * x, b = y * y, ea = fmaf(x, x, -a), eb = fmaf(y, y, -b);
    const float s = a + b, bb = s - a, e = (a - (s - bb)) + (b - bb);
    hi = s; lo = e + (ea + eb);
  }
  // sum over aligned groups of W lanes (every lane of a group ends with the group's sum)
  template <int W = 32> __device__ __forceinline__ void shfl_sum() {
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) {
      const float h = __shfl_xor_sync(0xffffffffu, hi, o), l = __shfl_xor_sync(0xffffffffu, lo, o);
      add(h, l);
    }
  }
  // += (a_hi, a_lo) without renormalising: the exact TwoSum of the high words, and the
  // low words (each ~2^-24 of the high ones) plus its error summed in FP32; two fewer
  // dependent operations per add, for reductions where the pair is only read at the end
  __device__ __forceinline__ void add_nr(float a, float b) {
    const float s = hi + a, bb = s - hi, e = (hi - (s - bb)) + (a - bb);
    hi = s; lo = (lo + b) + e;
  }
  __device__ __forceinline__ void add_nr(const NAcc& o) { add_nr(o.hi, o.lo); }
  __device__ __forceinline__ void shfl_sum_nr() {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float h = __shfl_xor_sync(0xffffffffu, hi, o), l = __shfl_xor_sync(0xffffffffu, lo, o);
      add_nr(h, l);
    }
  }
  __device__ __forceinline__ float value() const { return hi + lo; }
};
template <> struct NAcc<double> {
  double v = 0.0;
  __device__ __forceinline__ void add(double a, double b) { v += a + b; }
  __device__ __forceinline__ void add_sq(double x) { v = fma(x, x, v); }
  __device__ __forceinline__ void add(const NAcc& o) { v += o.v; }
  template <int W = 32> __device__ __forceinline__ void shfl_sum() {
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
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
constexpr int SLOTS = KBMAX;              // column slots per message (padded)

template <typename T> __device__ __forceinline__ cx<T> shfl_cx(cx<T> v, int src) {
  return mk<T>(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}
__device__ __forceinline__ void st_async_16(uint32_t addr, float4 v, uint32_t mbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];"
               ::"r"(addr), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "r"(mbar) : "memory");
}
__device__ __forceinline__ void st_async_8(uint32_t addr, float2 v, uint32_t mbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];"
               ::"r"(addr), "f"(v.x), "f"(v.y), "r"(mbar) : "memory");
}
__device__ __forceinline__ void st_async_16(uint32_t addr, double2 v, uint32_t mbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f64 [%0], {%1, %2}, [%3];"
               ::"r"(addr), "d"(v.x), "d"(v.y), "r"(mbar) : "memory");
}

// reflector scalars (zlarfg convention) from ||x||^2 below the pivot and alpha, with a
// correctly rounded square root and tau, scale within about one unit in the last place of
// correctly rounded (reciprocal forms, as LAPACK's own): the unitarity of
// H = I - tau v v^dag rests on tau and scale agreeing with ||v|| to working precision
template <typename T>
__device__ __forceinline__ void reflector(T xn2, T alr, T ali, T& beta, T& tr, T& ti, T& sr, T& si) {
  beta = alr; tr = ti = sr = si = T(0);
  // A column whose squared norm is below the normal range (noise of a rank-deficient
  // block) is left as is: tau = 0, H = I, which is exactly unitary.
  const T tot = alr * alr + ali * ali + xn2;
  if (!(xn2 == T(0) && ali == T(0)) && tot > T(16) * std::numeric_limits<T>::min()) {
    const T nrm = sqrt(tot);
    beta = alr >= T(0) ? -nrm : nrm;
    const T dr = alr - beta, di = ali;
    // |alpha - beta|^2 <= 4 tot: below the overflow edge, 1/beta and 1/|alpha - beta|^2 in
    // parallel give tau and scale by products (two divisions off each other's path instead
    // of five in a chain; on B300 each FP64 division is a long FP64 sequence); near it,
    // the divisions one by one with scale = 1 / (alpha - beta) by Smith's division
    // (|alr - beta| >= |ali|)
    if (tot < T(0.25) * std::numeric_limits<T>::max()) {
      const T rb = T(1) / beta, q = T(1) / (dr * dr + di * di);
      tr = -dr * rb;
      ti = -ali * rb;
      sr = dr * q;
      si = -di * q;
    } else {
      tr = (beta - alr) / beta;
      ti = -ali / beta;
      const T rt = di / dr, den = dr + di * rt;
      sr = T(1) / den; si = -rt / den;
    }
  }
}

// The same scalars for the complex64 register panel with one division on the critical
// path: 1/beta and 1/|alpha - beta|^2 in parallel, tau and scale by products (about one
// unit in the last place from correctly rounded, as LAPACK's own reciprocal forms). When
// |alpha - beta|^2 could overflow the Smith form above is used.
__device__ __forceinline__ void reflector_rf(float xn2, float alr, float ali, float& beta, float& tr, float& ti,
                                             float& sr, float& si) {
  const float tot = alr * alr + ali * ali + xn2;
  if (!(tot < 1e37f)) { reflector<float>(xn2, alr, ali, beta, tr, ti, sr, si); return; }
  beta = alr; tr = ti = sr = si = 0.f;
  if (!(xn2 == 0.f && ali == 0.f) && tot > 16.f * std::numeric_limits<float>::min()) {
    const float nrm = sqrtf(tot);
    beta = alr >= 0.f ? -nrm : nrm;
    const float dr = alr - beta, di = ali;
    const float rb = 1.f / beta, q = 1.f / fmaf(dr, dr, di * di);
    tr = -dr * rb;
    ti = -ali * rb;
    sr = dr * q;
    si = -di * q;
  }
}

template <typename T> struct __align__(16) VXp { cx<T> v, x; };

template <typename T> struct PanelSmem {
  static constexpr int HDR = 16;
  static constexpr int MSG = HDR + SLOTS * (int)sizeof(cx<T>);
  static constexpr size_t fixed(int nw) {
    return a16(2 * 16 * MSG)                               // recv [2][16]
         + a16(2 * SLOTS * sizeof(cx<T>))                  // pivot row copies [2]
         + a16((size_t)nw * 16)                            // per-warp norm partials
         + a16((size_t)nw * SLOTS * sizeof(cx<T>))         // per-warp slot partials
         + 3 * a16(KBMAX * sizeof(cx<T>))                  // tau, scale, beta
         + a16(KBMAX * (KBMAX + 1) * sizeof(cx<T>))        // g, then T
         + a16(2 * (SLOTS + 2) * sizeof(cx<T>))            // broadcast: cw[32], scale, tau
         + 64;
  }
};
// local rows: the panel's first kb rows (every CTA) followed by this CTA's slab
template <typename T> __host__ __device__ inline size_t panel_smem_bytes(int rps, int kb) {
  const size_t rows = (size_t)kb + rps;
  return a16(rows * (kb + 1) * sizeof(cx<T>)) + a16(rows * 2 * sizeof(cx<T>)) + PanelSmem<T>::fixed(PT / 32);
}
// Shared-memory blocks common to both panel kernels, carved after the row storage in
// the order PanelSmem::fixed counts them.
template <typename T> struct PanelShared {
  unsigned char* recvm; cx<T>* pivb; T* wpn; cx<T>* wps;
  cx<T>* taus; cx<T>* scl; cx<T>* bet; cx<T>* Ts; cx<T>* bc; uint64_t* mb;
};
template <typename T> __device__ __forceinline__ PanelShared<T> carve_panel_shared(unsigned char* q, int nw) {
  using L = PanelSmem<T>;
  PanelShared<T> sh;
  sh.recvm = q; q += a16(2 * 16 * L::MSG);
  sh.pivb = reinterpret_cast<cx<T>*>(q); q += a16(2 * SLOTS * sizeof(cx<T>));
  sh.wpn = reinterpret_cast<T*>(q); q += a16((size_t)nw * 16);
  sh.wps = reinterpret_cast<cx<T>*>(q); q += a16((size_t)nw * SLOTS * sizeof(cx<T>));
  sh.taus = reinterpret_cast<cx<T>*>(q); q += a16(KBMAX * sizeof(cx<T>));
  sh.scl = reinterpret_cast<cx<T>*>(q); q += a16(KBMAX * sizeof(cx<T>));
  sh.bet = reinterpret_cast<cx<T>*>(q); q += a16(KBMAX * sizeof(cx<T>));
  sh.Ts = reinterpret_cast<cx<T>*>(q); q += a16(KBMAX * (KBMAX + 1) * sizeof(cx<T>));
  sh.bc = reinterpret_cast<cx<T>*>(q); q += a16(2 * (SLOTS + 2) * sizeof(cx<T>));
  sh.mb = reinterpret_cast<uint64_t*>(q);
  return sh;
}

// Phases 3 and 4 of column jn. On entry (after a CTA barrier) each warp's norm partial
// is in wpn and its slot partials in wps; prow is this CTA's copy of panel row jn. On
// exit (after a CTA barrier) bc[buf] holds conj(tau) w_c for every column and the
// reflector's scale, and tau, scale, beta and the Gram values of column jn are stored.
template <typename T, int NW>
__device__ __forceinline__ void panel_exchange(const PanelShared<T>& sh, const cx<T>* prow, int jn, int kb,
                                               int rank, int CS, unsigned* err, bool& ok) {
  using L = PanelSmem<T>;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const cx<T> zero = mk<T>(0, 0);
  const uint32_t txb = (uint32_t)(CS * L::MSG);
  // ---- 3. exchange: every warp forms the CTA's message (the warps' partials summed)
  //      and pushes it to its share of the ranks (r = warp, warp + NW, ...), so the
  //      remote stores issue in parallel; warp 0 also copies the pivot row and arms
  //      this CTA's barrier
  const int buf = jn & 1;
  {
    cx<T> s = zero;
#pragma unroll
    for (int w = 0; w < NW; ++w) s = cadd<T>(s, sh.wps[w * SLOTS + lane]);
    NAcc<T> n;
    {
      const int w = lane & (NW - 1);  // each group of NW lanes holds every warp's partial
      if constexpr (std::is_same<T, float>::value) n.add(sh.wpn[w * 4], sh.wpn[w * 4 + 1]);
      else n.add(sh.wpn[w * 2], T(0));
    }
    n.template shfl_sum<NW>();
    cx<T> h;
    if constexpr (std::is_same<T, float>::value) h = mk<T>(n.hi, n.lo); else h = mk<T>(n.value(), 0);
    if (warp == 0) {
      sh.pivb[buf * SLOTS + lane] = prow[min(lane, kb - 1)];
      __syncwarp();
      if (lane == 0) mbar_arm(&sh.mb[buf], txb);  // release: the pivot copy is visible to the waiters
    }
    const uint32_t mine = smem_addr(sh.recvm + (buf * 16 + rank) * L::MSG);
    const uint32_t mbl = smem_addr(&sh.mb[buf]);
    if constexpr (std::is_same<T, float>::value) {
      // 17 chunks of 16 bytes: (norm hi, lo, 0, 0), then slot pairs
      const cx<T> sa = shfl_cx<T>(s, (2 * lane + 30) & 31), sb = shfl_cx<T>(s, (2 * lane + 31) & 31);
      const float4 ch = lane == 0 ? make_float4(h.x, h.y, 0.f, 0.f) : make_float4(sa.x, sa.y, sb.x, sb.y);
      if (lane < 17)
        for (int r = warp; r < CS; r += NW) st_async_16(map_rank(mine + 16 * lane, r), ch, map_rank(mbl, r));
    } else {
      for (int r = warp; r < CS; r += NW) {
        const uint32_t rb = map_rank(mine, r), rm = map_rank(mbl, r);
        st_async_16(rb + 16 + 16 * lane, s, rm);
        if (lane == 0) st_async_16(rb, h, rm);
      }
    }
  }
  if (warp == 0) {
    if (!mbar_wait_cl(&sh.mb[buf], (uint32_t)((jn >> 1) & 1))) ok = false;
    const cx<T>* piv = sh.pivb + buf * SLOTS;
    NAcc<T> ns;
    if ((lane & 15) < CS) {  // both half-warps hold every rank's norm partial
      const T* hh = reinterpret_cast<const T*>(sh.recvm + (buf * 16 + (lane & 15)) * L::MSG);
      ns.add(hh[0], hh[1]);
    }
    cx<T> S;
    {
      // all ranks' slots loaded at once (a fixed, predicated unroll), then a sum tree
      const unsigned char* base = sh.recvm + buf * 16 * L::MSG + L::HDR + min(lane, kb - 1) * sizeof(cx<T>);
      cx<T> v[16];
#pragma unroll
      for (int r = 0; r < 16; ++r) v[r] = r < CS ? *reinterpret_cast<const cx<T>*>(base + r * L::MSG) : zero;
#pragma unroll
      for (int h = 8; h > 0; h >>= 1)
#pragma unroll
        for (int r = 0; r < h; ++r) v[r] = cadd<T>(v[r], v[r + h]);
      S = v[0];
    }
    const cx<T> pc = piv[min(lane, kb - 1)];
    const cx<T> alpha = piv[jn];
    ns.template shfl_sum<16>();
    T beta, tr, ti, sr, si;
    reflector(ns.value(), alpha.x, alpha.y, beta, tr, ti, sr, si);
    if (lane == 0 && rank == 0 && !(isfinite(beta) && isfinite(sr) && isfinite(si)))
      atomicOr(err, DEVERR_NUMERIC);
    const cx<T> sc = mk<T>(sr, si), tau = mk<T>(tr, ti);
    const bool u = lane > jn && lane < kb;
    const cx<T> cwl = u ? cmul<T>(cconj<T>(tau), cadd<T>(pc, cmul<T>(cconj<T>(sc), S))) : zero;
    if (lane < jn) {
      const cx<T> gv = cmul<T>(cconj<T>(sh.scl[lane]), cadd<T>(cconj<T>(pc), cmul<T>(sc, cconj<T>(S))));
      sh.Ts[lane * (KBMAX + 1) + jn] = gv;
    }
    cx<T>* bb = sh.bc + buf * (SLOTS + 2);
    bb[lane] = cwl;
    if (lane == 0) { bb[SLOTS] = sc; sh.taus[jn] = tau; sh.scl[jn] = sc; sh.bet[jn] = mk<T>(beta, 0); }
  }
  asm volatile("bar.sync 1, %0;" ::"n"(NW * 32) : "memory");
}

// Compact-WY T of the panel (and tau) into global memory, from the Gram values and tau
// the column loop left in shared memory; run by one CTA of the cluster.
template <typename T, int NW>
__device__ __forceinline__ void panel_t_factor(const PanelShared<T>& sh, int kb, const PanelArgs<T>& a) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const cx<T> zero = mk<T>(0, 0);
  const long long k0 = a.k0;
  // compact-WY T (the last rank, whose slab is the shortest): with U the strict upper
  // part of V^dag V (held in sh.Ts), T^{-1} = diag(1/tau) + U, so column j of T solves
  // t_i = tau_i (delta_ij - sum_{k > i} U_ik t_k), i = j, j-1, ..., 0; this form also
  // covers tau_i = 0 (H_i = I, row i of T zero). Warp w takes columns w, w + NW, ...,
  // lane = row; each step finalises t_k on lane k and broadcasts it.
  constexpr int CPW = (KBMAX + NW - 1) / NW;
  cx<T> acc[CPW], t[CPW];
#pragma unroll
  for (int c = 0; c < CPW; ++c) { acc[c] = zero; t[c] = zero; }
  const cx<T> tau_l = lane < kb ? sh.taus[lane] : zero;
  for (int k = kb - 1; k >= 0; --k) {
    const cx<T> uk = lane < k ? sh.Ts[lane * (KBMAX + 1) + k] : zero;
#pragma unroll
    for (int c = 0; c < CPW; ++c) {
      const int j = warp + c * NW;
      if (k <= j && j < kb) {  // warp-uniform
        if (lane == k) t[c] = cmul<T>(tau_l, csub<T>(mk<T>(k == j ? T(1) : T(0), T(0)), acc[c]));
        const cx<T> tk = shfl_cx<T>(t[c], k);
        cfma<T>(acc[c], uk, tk);  // uk = 0 on lanes >= k
      }
    }
  }
#pragma unroll
  for (int c = 0; c < CPW; ++c) {
    const int j = warp + c * NW;
    if (j < kb && lane < kb) a.Tf[lane * a.ldt + j] = t[c];  // t = 0 below the diagonal
  }
  if (tid < kb) a.tau[k0 + tid] = sh.taus[tid];
}

template <typename T>
__global__ void __launch_bounds__(PT) k_qr_panel(PanelArgs<T> a) {
  constexpr int NT = PT;
  using L = PanelSmem<T>;
  pdl_launch_dependents();
  pdl_wait();
  constexpr int NW = NT / 32;
  extern __shared__ __align__(16) unsigned char sm[];
  cg::cluster_group cl = cg::this_cluster();
  const int CS = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int kb = a.kb, ldp = kb + 1, rps = a.rps;
  const int mr = a.m - a.k0;
  const int s0 = kb + rank * rps;                           // first slab row (panel index)
  const int nslab = max(0, min(rps, mr - s0));
  const int nloc = kb + nslab;
  const int rpw = (nloc + NW - 1) / NW;
  const int p0 = min(nloc, warp * rpw), p1 = min(nloc, p0 + rpw);
  const bool top_counts = rank == 0;                        // top rows enter rank 0's sums only
  auto grow = [&](int p) { return p < kb ? p : s0 + (p - kb); };

  unsigned char* q = sm;
  cx<T>* P = reinterpret_cast<cx<T>*>(q); q += a16((size_t)(kb + rps) * ldp * sizeof(cx<T>));
  // per row: v of the reflector being applied and x of the next pivot column, side by side
  // so that phase 2 reads both with one broadcast load
  VXp<T>* VX = reinterpret_cast<VXp<T>*>(q); q += a16((size_t)(kb + rps) * sizeof(VXp<T>));
  const PanelShared<T> sh = carve_panel_shared<T>(q, NW);
  uint64_t* mb = sh.mb;
  cx<T>* wps = sh.wps; T* wpn = sh.wpn;
  cx<T>* scl = sh.scl; cx<T>* bet = sh.bet; cx<T>* bc = sh.bc;

  const long long k0 = a.k0;
  if (tid == 0) {
    mbar_init1(&mb[0]);
    mbar_init1(&mb[1]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // load: lane = column, this warp's rows, all copies in flight (cp.async, no registers)
  if (lane < kb) {
    for (int p = p0; p < p1; ++p) {
      const cx<T>* src = a.A + (k0 + grow(p)) * a.lda + k0 + lane;
      asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_addr(P + p * ldp + lane)),
                   "l"(src), "n"((int)sizeof(cx<T>)) : "memory");
    }
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  cl.sync();  // every CTA's barriers exist before anyone sends; panel loaded
  bool ok = true;

  const cx<T> zero = mk<T>(0, 0);
  cx<T> scale = zero, cw = zero, cwn = zero;

  for (int jn = 0; jn < kb; ++jn) {
    const int jp = jn - 1;
    // local index = panel row for the top block, and g(p) is increasing in p
    const int plo = max(p0, min(p1, max(jp, 0)));
    // ---- 1. lane = row
    NAcc<T> nacc;
    for (int p = plo + lane; p < p1; p += 64) {
      const bool two = p + 32 < p1;
      cx<T> r0 = P[p * ldp + jn], r1 = zero, u0 = zero, u1 = zero;
      if (jp >= 0) u0 = P[p * ldp + jp];
      if (two) { r1 = P[(p + 32) * ldp + jn]; if (jp >= 0) u1 = P[(p + 32) * ldp + jp]; }
      cx<T> v0 = zero, v1 = zero;
      if (jp >= 0) { v0 = (p == jp) ? mk<T>(1, 0) : cmul<T>(scale, u0); v1 = cmul<T>(scale, u1); }
      r0 = csub<T>(r0, cmul<T>(v0, cwn));
      r1 = csub<T>(r1, cmul<T>(v1, cwn));
      P[p * ldp + jn] = r0; VX[p] = VXp<T>{v0, r0};
      if (p > jn && (top_counts || p >= kb)) { nacc.add_sq(r0.x); nacc.add_sq(r0.y); }
      if (two) {
        P[(p + 32) * ldp + jn] = r1; VX[p + 32] = VXp<T>{v1, r1};
        if (p + 32 > jn && (top_counts || p + 32 >= kb)) { nacc.add_sq(r1.x); nacc.add_sq(r1.y); }
      }
    }
    __syncwarp();
    // ---- 2. lane = column
    const int col = (lane < kb) ? lane : jn;
    const bool upd = lane > jn && lane < kb;
    const int slo = max(plo, min(p1, jn + 1));
    const int alo = top_counts ? slo : max(slo, min(p1, kb));
    {
      // rows that take the update only (the replicated pivot rows outside rank 0's sums):
      // four rows' loads ahead of their stores
      int p = plo;
      for (; p + 3 < alo; p += 4) {
        cx<T> y[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) y[u] = csub<T>(P[(p + u) * ldp + col], cmul<T>(VX[p + u].v, cw));
        if (upd) {
#pragma unroll
          for (int u = 0; u < 4; ++u) P[(p + u) * ldp + col] = y[u];
        }
      }
      for (; p < alo; ++p) {
        const cx<T> y = csub<T>(P[p * ldp + col], cmul<T>(VX[p].v, cw));
        if (upd) P[p * ldp + col] = y;
      }
    }
    cx<T> acc0 = zero, acc1 = zero;
    int p = alo;
    for (; p + 3 < p1; p += 4) {
      cx<T> v[4], x[4], y[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const VXp<T> t = VX[p + u];
        v[u] = t.v; x[u] = t.x; y[u] = P[(p + u) * ldp + col];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) y[u] = csub<T>(y[u], cmul<T>(v[u], cw));
      if (upd) {
#pragma unroll
        for (int u = 0; u < 4; ++u) P[(p + u) * ldp + col] = y[u];
      }
      cfma<T>(acc0, cconj<T>(x[0]), y[0]);
      cfma<T>(acc1, cconj<T>(x[1]), y[1]);
      cfma<T>(acc0, cconj<T>(x[2]), y[2]);
      cfma<T>(acc1, cconj<T>(x[3]), y[3]);
    }
    for (; p < p1; ++p) {
      const VXp<T> t = VX[p];
      const cx<T> v0 = t.v, x0 = t.x;
      const cx<T> y0 = csub<T>(P[p * ldp + col], cmul<T>(v0, cw));
      if (upd) P[p * ldp + col] = y0;
      cfma<T>(acc0, cconj<T>(x0), y0);
    }
    nacc.shfl_sum();
    wps[warp * SLOTS + lane] = cadd<T>(acc0, acc1);
    if (lane == 0) {
      if constexpr (std::is_same<T, float>::value) { wpn[warp * 4 + 0] = nacc.hi; wpn[warp * 4 + 1] = nacc.lo; }
      else { wpn[warp * 2 + 0] = nacc.value(); wpn[warp * 2 + 1] = 0; }
    }
    __syncthreads();
    panel_exchange<T, NW>(sh, P + jn * ldp, jn, kb, rank, CS, a.err, ok);
    const int buf = jn & 1;
    {
      const cx<T>* bb = bc + buf * (SLOTS + 2);
      scale = bb[SLOTS];
      cw = bb[lane];
      cwn = (jn + 1 < kb) ? bb[jn + 1] : zero;
    }
  }
  if (!ok && tid == 0) atomicOr(a.err, DEVERR_TIMEOUT);
  __syncthreads();

  if (rank == CS - 1) panel_t_factor<T, NW>(sh, kb, a);
  // ---- V (v = scale * raw column below the pivot, unit diagonal) and R / zeros into A;
  //      lane = column, the top block from rank 0 only
  if (lane < kb) {
    const cx<T> sc = scl[lane], bc = bet[lane];
    const int pstart = (rank == 0) ? p0 : max(p0, kb);
    auto put = [&](int p, cx<T> pv) {
      const int g = grow(p);
      a.V[(k0 + g) * a.ldv + k0 + lane] = (g == lane) ? mk<T>(1, 0) : (g > lane ? cmul<T>(sc, pv) : zero);
      a.A[(k0 + g) * a.lda + k0 + lane] = (lane > g) ? pv : (lane == g ? bc : zero);
    };
    int p = pstart;
    for (; p + 3 < p1; p += 4) {  // four rows' loads ahead of their stores
      cx<T> pv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) pv[u] = P[(p + u) * ldp + lane];
#pragma unroll
      for (int u = 0; u < 4; ++u) put(p + u, pv[u]);
    }
    for (; p < p1; ++p) put(p, P[p * ldp + lane]);
  }
  cl.sync();
}

// Grid form of the complex128 panel. Its cost is the FP64 work of each CTA (~230 cycles per
// row and column on B300's FP64 pipe), so for tall panels many CTAs with few slab rows beat
// one cluster of at most 16: a cooperative launch of G CTAs, the local phases of k_qr_panel
// unchanged (every CTA holds the kb pivot rows and its slab), and per column one exchange
// through global memory in place of the cluster's remote stores: each CTA writes its
// partial sums (the 32 slots and the norm) to part[parity][cta], a grid barrier (bounded
// wait), then every CTA adds the G partials in the same order and forms the same reflector.
// The parity double buffer lets the next column's writes go ahead while slower CTAs still
// read this column's sums.
template <typename T, int NW>
__device__ __forceinline__ void panel_exchange_g(const PanelShared<T>& sh, const cx<T>* prow, int jn, int kb,
                                                 int rank, int G, cx<T>* part, unsigned* bar, unsigned* err,
                                                 bool& ok) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const cx<T> zero = mk<T>(0, 0);
  const int buf = jn & 1;
  constexpr int PS = SLOTS + 1;  // a CTA's record: 32 slots, then the norm
  if (warp == 0) {
    cx<T> s = zero;
#pragma unroll
    for (int w = 0; w < NW; ++w) s = cadd<T>(s, sh.wps[w * SLOTS + lane]);
    T nrm = T(0);
#pragma unroll
    for (int w = 0; w < NW; ++w) nrm += sh.wpn[w * 2];
    cx<T>* mine = part + ((long long)buf * G + rank) * PS;
    mine[lane] = s;
    if (lane == 0) mine[SLOTS] = mk<T>(nrm, T(0));
    sh.pivb[buf * SLOTS + lane] = prow[min(lane, kb - 1)];
  }
  if (!grid_barrier(bar, (unsigned)G, err)) ok = false;
  // the G records summed in a fixed order, identical in every CTA: warp w loads the records
  // of CTAs w, w + NW, ... at once (lane = slot, lane 0 also the norm) and adds them in
  // order, then warp 0 adds the warps' sums in order
  if (ok) {
    constexpr int PW = (PG_MAX + NW - 1) / NW;
    const cx<T>* all = part + (long long)buf * G * PS;
    cx<T> v[PW];
    T nv[PW];
#pragma unroll
    for (int i = 0; i < PW; ++i) {
      const int g = warp + NW * i;
      v[i] = g < G ? __ldcg(all + (long long)g * PS + lane) : zero;
      nv[i] = (g < G && lane == 0) ? __ldcg(all + (long long)g * PS + SLOTS).x : T(0);
    }
    // pairwise, so that the FP64 adds form a tree of depth log2(PW) rather than a chain
#pragma unroll
    for (int h = 1; h < PW; h *= 2)
#pragma unroll
      for (int i = 0; i + h < PW; i += 2 * h) { v[i] = cadd<T>(v[i], v[i + h]); nv[i] += nv[i + h]; }
    sh.wps[warp * SLOTS + lane] = v[0];  // the CTA's own partials were read before the barrier
    if (lane == 0) sh.wpn[warp * 2] = nv[0];
  }
  __syncthreads();
  if (warp == 0 && ok) {
    cx<T> vw[NW];
    T nw[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) { vw[w] = sh.wps[w * SLOTS + lane]; nw[w] = sh.wpn[w * 2]; }
#pragma unroll
    for (int h = 1; h < NW; h *= 2)
#pragma unroll
      for (int w = 0; w + h < NW; w += 2 * h) { vw[w] = cadd<T>(vw[w], vw[w + h]); nw[w] += nw[w + h]; }
    const cx<T> S = vw[0];
    const T ns = nw[0];
    const cx<T>* piv = sh.pivb + buf * SLOTS;
    const cx<T> pc = piv[min(lane, kb - 1)];
    const cx<T> alpha = piv[jn];
    T beta, tr, ti, sr, si;
    reflector(ns, alpha.x, alpha.y, beta, tr, ti, sr, si);
    if (lane == 0 && rank == 0 && !(isfinite(beta) && isfinite(sr) && isfinite(si)))
      atomicOr(err, DEVERR_NUMERIC);
    const cx<T> sc = mk<T>(sr, si), tau = mk<T>(tr, ti);
    const bool u = lane > jn && lane < kb;
    const cx<T> cwl = u ? cmul<T>(cconj<T>(tau), cadd<T>(pc, cmul<T>(cconj<T>(sc), S))) : zero;
    if (lane < jn) {
      const cx<T> gv = cmul<T>(cconj<T>(sh.scl[lane]), cadd<T>(cconj<T>(pc), cmul<T>(sc, cconj<T>(S))));
      sh.Ts[lane * (KBMAX + 1) + jn] = gv;
    }
    cx<T>* bb = sh.bc + buf * (SLOTS + 2);
    bb[lane] = cwl;
    if (lane == 0) { bb[SLOTS] = sc; sh.taus[jn] = tau; sh.scl[jn] = sc; sh.bet[jn] = mk<T>(beta, 0); }
  }
  __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(PT) k_qr_panel_g(PanelArgs<T> a, cx<T>* part, unsigned* bar) {
  constexpr int NT = PT;
  using L = PanelSmem<T>;
  pdl_launch_dependents();
  pdl_wait();
  constexpr int NW = NT / 32;
  extern __shared__ __align__(16) unsigned char sm[];
  const int CS = (int)gridDim.x;
  const int rank = (int)blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int kb = a.kb, ldp = kb + 1, rps = a.rps;
  const int mr = a.m - a.k0;
  const int s0 = kb + rank * rps;                           // first slab row (panel index)
  const int nslab = max(0, min(rps, mr - s0));
  const int nloc = kb + nslab;
  const int rpw = (nloc + NW - 1) / NW;
  const int p0 = min(nloc, warp * rpw), p1 = min(nloc, p0 + rpw);
  const bool top_counts = rank == 0;                        // top rows enter rank 0's sums only
  auto grow = [&](int p) { return p < kb ? p : s0 + (p - kb); };

  unsigned char* q = sm;
  cx<T>* P = reinterpret_cast<cx<T>*>(q); q += a16((size_t)(kb + rps) * ldp * sizeof(cx<T>));
  // per row: v of the reflector being applied and x of the next pivot column, side by side
  // so that phase 2 reads both with one broadcast load
  VXp<T>* VX = reinterpret_cast<VXp<T>*>(q); q += a16((size_t)(kb + rps) * sizeof(VXp<T>));
  const PanelShared<T> sh = carve_panel_shared<T>(q, NW);
  cx<T>* wps = sh.wps; T* wpn = sh.wpn;
  cx<T>* scl = sh.scl; cx<T>* bet = sh.bet; cx<T>* bc = sh.bc;

  const long long k0 = a.k0;
  // load: lane = column, this warp's rows, all copies in flight (cp.async, no registers)
  if (lane < kb) {
    for (int p = p0; p < p1; ++p) {
      const cx<T>* src = a.A + (k0 + grow(p)) * a.lda + k0 + lane;
      asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_addr(P + p * ldp + lane)),
                   "l"(src), "n"((int)sizeof(cx<T>)) : "memory");
    }
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
  bool ok = true;

  const cx<T> zero = mk<T>(0, 0);
  cx<T> scale = zero, cw = zero, cwn = zero;

  for (int jn = 0; jn < kb; ++jn) {
    const int jp = jn - 1;
    // local index = panel row for the top block, and g(p) is increasing in p
    const int plo = max(p0, min(p1, max(jp, 0)));
    // ---- 1. lane = row
    NAcc<T> nacc;
    for (int p = plo + lane; p < p1; p += 64) {
      const bool two = p + 32 < p1;
      cx<T> r0 = P[p * ldp + jn], r1 = zero, u0 = zero, u1 = zero;
      if (jp >= 0) u0 = P[p * ldp + jp];
      if (two) { r1 = P[(p + 32) * ldp + jn]; if (jp >= 0) u1 = P[(p + 32) * ldp + jp]; }
      cx<T> v0 = zero, v1 = zero;
      if (jp >= 0) { v0 = (p == jp) ? mk<T>(1, 0) : cmul<T>(scale, u0); v1 = cmul<T>(scale, u1); }
      r0 = csub<T>(r0, cmul<T>(v0, cwn));
      r1 = csub<T>(r1, cmul<T>(v1, cwn));
      P[p * ldp + jn] = r0; VX[p] = VXp<T>{v0, r0};
      if (p > jn && (top_counts || p >= kb)) { nacc.add_sq(r0.x); nacc.add_sq(r0.y); }
      if (two) {
        P[(p + 32) * ldp + jn] = r1; VX[p + 32] = VXp<T>{v1, r1};
        if (p + 32 > jn && (top_counts || p + 32 >= kb)) { nacc.add_sq(r1.x); nacc.add_sq(r1.y); }
      }
    }
    __syncwarp();
    // ---- 2. lane = column
    const int col = (lane < kb) ? lane : jn;
    const bool upd = lane > jn && lane < kb;
    const int slo = max(plo, min(p1, jn + 1));
    const int alo = top_counts ? slo : max(slo, min(p1, kb));
    {
      // rows that take the update only (the replicated pivot rows outside rank 0's sums):
      // four rows' loads ahead of their stores
      int p = plo;
      for (; p + 3 < alo; p += 4) {
        cx<T> y[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) y[u] = csub<T>(P[(p + u) * ldp + col], cmul<T>(VX[p + u].v, cw));
        if (upd) {
#pragma unroll
          for (int u = 0; u < 4; ++u) P[(p + u) * ldp + col] = y[u];
        }
      }
      for (; p < alo; ++p) {
        const cx<T> y = csub<T>(P[p * ldp + col], cmul<T>(VX[p].v, cw));
        if (upd) P[p * ldp + col] = y;
      }
    }
    cx<T> acc0 = zero, acc1 = zero;
    int p = alo;
    for (; p + 3 < p1; p += 4) {
      cx<T> v[4], x[4], y[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const VXp<T> t = VX[p + u];
        v[u] = t.v; x[u] = t.x; y[u] = P[(p + u) * ldp + col];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) y[u] = csub<T>(y[u], cmul<T>(v[u], cw));
      if (upd) {
#pragma unroll
        for (int u = 0; u < 4; ++u) P[(p + u) * ldp + col] = y[u];
      }
      cfma<T>(acc0, cconj<T>(x[0]), y[0]);
      cfma<T>(acc1, cconj<T>(x[1]), y[1]);
      cfma<T>(acc0, cconj<T>(x[2]), y[2]);
      cfma<T>(acc1, cconj<T>(x[3]), y[3]);
    }
    for (; p < p1; ++p) {
      const VXp<T> t = VX[p];
      const cx<T> v0 = t.v, x0 = t.x;
      const cx<T> y0 = csub<T>(P[p * ldp + col], cmul<T>(v0, cw));
      if (upd) P[p * ldp + col] = y0;
      cfma<T>(acc0, cconj<T>(x0), y0);
    }
    nacc.shfl_sum();
    wps[warp * SLOTS + lane] = cadd<T>(acc0, acc1);
    if (lane == 0) {
      if constexpr (std::is_same<T, float>::value) { wpn[warp * 4 + 0] = nacc.hi; wpn[warp * 4 + 1] = nacc.lo; }
      else { wpn[warp * 2 + 0] = nacc.value(); wpn[warp * 2 + 1] = 0; }
    }
    __syncthreads();
    panel_exchange_g<T, NW>(sh, P + jn * ldp, jn, kb, rank, CS, part, bar, a.err, ok);
    if (!ok) break;  // a grid barrier ran out: every CTA's next wait will too
    const int buf = jn & 1;
    {
      const cx<T>* bb = bc + buf * (SLOTS + 2);
      scale = bb[SLOTS];
      cw = bb[lane];
      cwn = (jn + 1 < kb) ? bb[jn + 1] : zero;
    }
  }
  if (!ok && tid == 0) atomicOr(a.err, DEVERR_TIMEOUT);
  __syncthreads();

  if (rank == CS - 1) panel_t_factor<T, NW>(sh, kb, a);
  // ---- V (v = scale * raw column below the pivot, unit diagonal) and R / zeros into A;
  //      lane = column, the top block from rank 0 only
  if (lane < kb) {
    const cx<T> sc = scl[lane], bc = bet[lane];
    const int pstart = (rank == 0) ? p0 : max(p0, kb);
    auto put = [&](int p, cx<T> pv) {
      const int g = grow(p);
      a.V[(k0 + g) * a.ldv + k0 + lane] = (g == lane) ? mk<T>(1, 0) : (g > lane ? cmul<T>(sc, pv) : zero);
      a.A[(k0 + g) * a.lda + k0 + lane] = (lane > g) ? pv : (lane == g ? bc : zero);
    };
    int p = pstart;
    for (; p + 3 < p1; p += 4) {  // four rows' loads ahead of their stores
      cx<T> pv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) pv[u] = P[(p + u) * ldp + lane];
#pragma unroll
      for (int u = 0; u < 4; ++u) put(p + u, pv[u]);
    }
    for (; p < p1; ++p) put(p, P[p * ldp + lane]);
  }
}


// Register-file form of the panel (complex64), used when each warp's share of the slab
// fits in RF_RPW rows of registers, lane = column; the replicated top kb rows stay in
// shared memory (every step needs the pivot row from there), split over the warps.
// It also takes the application of reflector j-1 to the trailing columns off the
// critical path: column j+1 of step j is computed alone (lane = row), and the partial
// sums go out against the columns as they were before reflector j-1,
//   S'_c = sum_{g > j} conj(x_g) P[g, c],   h = sum_{g > j} conj(x_g) x^{(j-1)}_g,
// from which the receiver forms S_c = S'_c - h scale_{j-1} conj(tau_{j-1}) w_c (one more
// scalar in the message header). The trailing update by reflector j-1 then runs while
// the messages are in flight. Arrays in shared memory: X (double-buffered), the raw pivot
// column x_j of every local row; Y, the slab values of the next pivot column, published
// by that lane during the trailing update. The coefficients cws = scale conj(tau) w_c of
// the lanes fold the reflector's scale into the update of the raw column. Warp 0 holds no
// rows: it waits for the messages and forms the reflector while warps 1..11 apply the
// trailing update, so that update leaves the critical path. The norm and h travel ahead
// of the slot sums: warp 0 reduces the row warps' lane partials during their pass B and
// pushes the CTA's 16-byte header on a barrier of its own, so the reflector scalars are
// formed while the slot messages are still in flight.
constexpr int RF_NT = 384;  // threads per CTA: the reflector warp and 11 row warps
constexpr int RF_RPW = 30;  // slab rows per row warp held in registers (11 x 30 = 330 per CTA)

template <typename T> __host__ __device__ inline size_t panel_rf_smem_bytes(int kb) {
  constexpr int slots = (RF_NT / 32 - 1) * RF_RPW;
  return a16((size_t)kb * (kb + 1) * sizeof(cx<T>)) + a16((size_t)(2 * (KBMAX + slots) + slots) * sizeof(cx<T>)) +
         a16((size_t)(RF_NT / 32 - 1) * 32 * 16) + 2 * 16 * 16 + PanelSmem<T>::fixed(RF_NT / 32);
}

// p - v c with every rounding fixed (four explicit FMAs), so that the trailing update and
// the column pass produce the same bits for the pivot column
__device__ __forceinline__ cx<float> upd_rn(cx<float> p, cx<float> v, cx<float> c) {
  return mk<float>(__fmaf_rn(-v.x, c.x, __fmaf_rn(v.y, c.y, p.x)), __fmaf_rn(-v.x, c.y, __fmaf_rn(-v.y, c.x, p.y)));
}
__device__ __forceinline__ cx<float> cmul_rn(cx<float> a, cx<float> b) {
  return mk<float>(__fmaf_rn(a.x, b.x, -__fmul_rn(a.y, b.y)), __fmaf_rn(a.x, b.y, __fmul_rn(a.y, b.x)));
}
__device__ __forceinline__ cx<float> sub_rn(cx<float> p, cx<float> c) {
  return mk<float>(__fsub_rn(p.x, c.x), __fsub_rn(p.y, c.y));
}

template <int RPW>
__global__ void __launch_bounds__(RF_NT, 1) k_qr_panel_rf(PanelArgs<float> a) {
  using T = float;
  constexpr int NT = RF_NT, NW = NT / 32, RW = NW - 1;  // warps 1 .. RW hold the rows
  static_assert(RW <= 16 && RPW <= 32 && RPW % 2 == 0,
                "one tree level per halving; one slab row per lane; slab rows in 16-byte pairs");
  constexpr int TPW = (KBMAX + RW - 1) / RW;          // top rows per row warp: t = rw + RW i
  pdl_launch_dependents();
  pdl_wait();
  extern __shared__ __align__(16) unsigned char sm[];
  cg::cluster_group cl = cg::this_cluster();
  const int CS = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int kb = a.kb, ldp = kb + 1, rps = a.rps;
  const int mr = a.m - a.k0;
  const int s0 = kb + rank * rps;                  // first slab row (panel index)
  const int nslab = max(0, min(rps, mr - s0));
  const int rw = warp - 1;                         // row-warp index; -1 for the reflector warp
  const int spw = (nslab + RW - 1) / RW;           // slab rows per row warp, <= RPW (host-checked)
  const int q0 = rw < 0 ? 0 : min(nslab, rw * spw);
  const int cnt = rw < 0 ? 0 : min(nslab, q0 + spw) - q0;  // this warp's slab rows q0 .. q0 + cnt - 1
  const int tcnt = rw < 0 ? 0 : TPW;               // top rows t = rw + RW i < kb, i < tcnt
  const bool top_counts = rank == 0;               // top rows enter rank 0's sums only
  // X: KBMAX top-row slots, then RPW slots per row warp (rows past cnt stay zero, so the
  // row loops below run over all RPW slots without guards, two rows per 16-byte access);
  // Y: RPW slots per row warp
  const int xs = KBMAX + RW * RPW;
  const int xb = rw < 0 ? 0 : rw * RPW;            // this warp's first slab slot

  unsigned char* q = sm;
  cx<T>* Pt = reinterpret_cast<cx<T>*>(q); q += a16((size_t)kb * ldp * sizeof(cx<T>));
  cx<T>* X = reinterpret_cast<cx<T>*>(q);
  cx<T>* Y = X + 2 * xs; q += a16((size_t)(2 * xs + RW * RPW) * sizeof(cx<T>));
  float4* pn = reinterpret_cast<float4*>(q); q += a16((size_t)RW * 32 * sizeof(float4));  // lane partials
  float* recvh = reinterpret_cast<float*>(q); q += 2 * 16 * 16;  // [2][16 ranks] headers (norm hi, lo, h)
  const PanelShared<T> sh = carve_panel_shared<T>(q, NW);
  const long long k0 = a.k0;
  const cx<T> zero = mk<T>(0, 0);
  uint64_t* mbh = sh.mb + 2;  // header barriers; sh.mb[0..1] count the slot messages
  if (tid == 0) {
    mbar_init1(&sh.mb[0]);
    mbar_init1(&sh.mb[1]);
    mbar_init1(&mbh[0]);
    mbar_init1(&mbh[1]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int i = tid; i < 2 * xs + RW * RPW; i += NT) X[i] = zero;
  __syncthreads();
  // load, lane = column: the top rows into shared memory (cp.async), the slab into registers
  if (lane < kb && rw >= 0)
    for (int t = rw; t < kb; t += RW)
      asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_addr(Pt + t * ldp + lane)),
                   "l"(a.A + (k0 + t) * a.lda + k0 + lane), "n"((int)sizeof(cx<T>)) : "memory");
  cx<T> R[RPW];
  {
    const cx<T>* src = a.A + (k0 + s0 + q0) * a.lda + k0 + min(lane, kb - 1);
#pragma unroll
    for (int r = 0; r < RPW; ++r) R[r] = (r < cnt && lane < kb) ? src[r * a.lda] : zero;
  }
  if (lane == 0 && rw >= 0) {
#pragma unroll
    for (int r = 0; r < RPW; ++r) Y[xb + r] = R[r];
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  cl.sync();  // every CTA's barriers exist before anyone sends; top rows and Y in place
  bool ok = true;
  constexpr int MSGS = SLOTS * (int)sizeof(cx<T>);      // a slot message: 32 slots of 8 bytes
  const uint32_t txs = (uint32_t)(CS * MSGS), txh = (uint32_t)(CS * 16);
  const int col = min(lane, kb - 1);
  cx<T> cw = zero, cws = zero;  // this lane's conj(tau) w_c of reflector j-1, and scale_{j-1} cw
  cx<T> cwj = zero, cwsj = zero;  // the same two for column jn, the step's pivot column

  for (int jn = 0; jn < kb; ++jn) {
    const int jp = jn - 1, buf = jn & 1;
    const cx<T>* Xp = X + ((jn + 1) & 1) * xs;  // raw column jp
    cx<T>* Xn = X + buf * xs;                   // raw column jn
    NAcc<T> nacc, nacc2;
    cx<T> hp = zero, hp2 = zero;
    // ---- A. column jn alone, lane = row (one slab row per lane, cnt <= 32, and lanes
    //      0 .. tcnt-1 one top row each, as two independent chains): x_jn = column jn after
    //      reflector jp; norm and h partials
    if (lane < cnt) {
      cx<T> x = Y[xb + lane];
      if (jp >= 0) {
        const cx<T> u = Xp[KBMAX + xb + lane];
        x = upd_rn(x, u, cwsj);
        cfma<T>(hp, cconj<T>(x), u);
      }
      Xn[KBMAX + xb + lane] = x;
      nacc.set_abs2(x.x, x.y);
    }
    if (lane < tcnt) {
      const int t = rw + RW * lane;
      if (t < kb) {
        cx<T> x = Pt[t * ldp + jn];
        if (jp >= 0 && t >= jp) x = (t == jp) ? sub_rn(x, cwj) : upd_rn(x, Xp[t], cwsj);
        Xn[t] = x;
        if (top_counts && t > jn) {
          nacc2.set_abs2(x.x, x.y);
          if (jp >= 0) cfma<T>(hp2, cconj<T>(x), Xp[t]);
        }
      }
    }
    nacc.add_nr(nacc2);
    hp = cadd<T>(hp, hp2);
    // the lane partials of the norm and of h go to the reflector warp, which sums them
    // while the row warps run pass B
    if (rw >= 0) {
      pn[rw * 32 + lane] = make_float4(nacc.hi, nacc.lo, hp.x, hp.y);
      asm volatile("bar.arrive 2, %0;" ::"n"(NT) : "memory");
    }
    __syncwarp();
    // ---- B. S'_c over this warp's rows below pivot jn, lane = column, the columns as they
    //      were before reflector jp; the owner of row jn copies it for the reflector
    cx<T> acc0 = zero, acc1 = zero;
    if (rw >= 0) {  // warp-uniform: the reflector warp skips the predicated row loops
      const float4* Xs = reinterpret_cast<const float4*>(Xn + KBMAX + xb);
      cx<T> acc2 = zero, acc3 = zero;
#pragma unroll
      for (int r = 0; r < RPW; r += 2) {
        const float4 e = Xs[r / 2];
        if ((r / 2) & 1) {
          cfma<T>(acc2, mk<T>(e.x, -e.y), R[r]);
          cfma<T>(acc3, mk<T>(e.z, -e.w), R[r + 1]);
        } else {
          cfma<T>(acc0, mk<T>(e.x, -e.y), R[r]);
          cfma<T>(acc1, mk<T>(e.z, -e.w), R[r + 1]);
        }
      }
      acc0 = cadd<T>(acc0, acc2);
      acc1 = cadd<T>(acc1, acc3);
    }
    if (top_counts) {
#pragma unroll
      for (int i = 0; i < TPW; ++i) {
        const int t = rw + RW * i;
        if (i < tcnt && t < kb && t > jn) cfma<T>(acc1, cconj<T>(Xn[t]), Pt[t * ldp + col]);
      }
    }
    if (rw == jn % RW) sh.pivb[buf * SLOTS + lane] = Pt[jn * ldp + col];
    if (rw >= 0) {
      sh.wps[warp * SLOTS + lane] = cadd<T>(acc0, acc1);
      // every row warp's slot partials and the pivot row copy are in place
      asm volatile("bar.sync 3, %0;" ::"n"(NT) : "memory");
      // ---- C. the row warps sum the CTA's slots and push them to their share of the
      //      ranks: 32 chunks of 8 bytes on the slot barrier
      {
        cx<T> s = zero;
#pragma unroll
        for (int w = 1; w < NW; ++w) s = cadd<T>(s, sh.wps[w * SLOTS + lane]);
        if (rw == 0 && lane == 0) mbar_arm(&sh.mb[buf], txs);
        const uint32_t mine = smem_addr(sh.recvm + (buf * 16 + rank) * MSGS);
        const uint32_t mbl = smem_addr(&sh.mb[buf]);
        // every lane sends its own slot (8 bytes)
        for (int r = rw; r < CS; r += RW) st_async_8(map_rank(mine + 8 * lane, r), make_float2(s.x, s.y), map_rank(mbl, r));
      }
      // ---- D. while the messages fly: reflector jp on the trailing columns (lanes c >= jn;
      //      cws = 0 elsewhere), in registers and on this warp's top rows; lane jn + 1
      //      publishes its slab values for the next step's column pass
      if (jp >= 0) {
        const float4* Vs = reinterpret_cast<const float4*>(Xp + KBMAX + xb);
#pragma unroll
        for (int r = 0; r < RPW; r += 2) {
          const float4 e = Vs[r / 2];
          R[r] = upd_rn(R[r], mk<T>(e.x, e.y), cws);
          R[r + 1] = upd_rn(R[r + 1], mk<T>(e.z, e.w), cws);
        }
#pragma unroll
        for (int i = 0; i < TPW; ++i) {
          const int t = rw + RW * i;
          if (i < tcnt && t < kb && t >= jp) {
            const cx<T> p = Pt[t * ldp + col];
            const cx<T> y = (t == jp) ? sub_rn(p, cw) : upd_rn(p, Xp[t], cws);
            if (lane >= jn && lane < kb) Pt[t * ldp + lane] = y;
          }
        }
      }
      if (lane == jn + 1) {
#pragma unroll
        for (int r = 0; r < RPW; ++r)
          if (r % 2 == 0)
            reinterpret_cast<float4*>(Y + xb)[r / 2] = make_float4(R[r].x, R[r].y, R[r + 1].x, R[r + 1].y);
      }
    } else {
      // ---- the reflector warp. The CTA's norm (double-float) and h from the lane partials
      //      (during pass B), pushed at once to every rank on the header barrier
      asm volatile("bar.sync 2, %0;" ::"n"(NT) : "memory");
      NAcc<T> nw[RW];
      float hxw[RW], hyw[RW];
#pragma unroll
      for (int w = 0; w < RW; ++w) {
        const float4 e = pn[w * 32 + lane];
        nw[w].hi = e.x; nw[w].lo = e.y; hxw[w] = e.z; hyw[w] = e.w;
      }
#pragma unroll
      for (int h = 8; h > 0; h >>= 1)  // tree over the row warps (RW <= 16)
#pragma unroll
        for (int w = 0; w < h; ++w)
          if (w + h < RW) { nw[w].add_nr(nw[w + h]); hxw[w] += hxw[w + h]; hyw[w] += hyw[w + h]; }
      NAcc<T> n0 = nw[0];
      float hx = hxw[0], hy = hyw[0];
      n0.shfl_sum_nr();
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        hx += __shfl_xor_sync(0xffffffffu, hx, o);
        hy += __shfl_xor_sync(0xffffffffu, hy, o);
      }
      if (lane == 0) mbar_arm(&mbh[buf], txh);
      if (lane < CS)
        st_async_16(map_rank(smem_addr(recvh + (buf * 16 + rank) * 4), lane), make_float4(n0.hi, n0.lo, hx, hy),
                    map_rank(smem_addr(&mbh[buf]), lane));
      asm volatile("bar.sync 3, %0;" ::"n"(NT) : "memory");
      // ---- E. the pivot row (copied in pass B), alpha and the Gram scales; then all ranks'
      //      headers and the reflector scalars while the slot messages are still in flight;
      //      then the slots, the correction by h and conj(tau) w_c
      cx<T> pc = sh.pivb[buf * SLOTS + col];
      if (jp >= 0) pc = upd_rn(pc, Xp[jn], cws);
      const cx<T> alpha = shfl_cx<T>(pc, jn);
      const cx<T> scl_l = lane < jn ? sh.scl[lane] : zero;
      if (!mbar_wait_cl(&mbh[buf], (uint32_t)((jn >> 1) & 1))) ok = false;
      NAcc<T> ns;
      float hxs = 0.f, hys = 0.f;
      if ((lane & 15) < CS) {  // lane r of each half-warp holds rank r's header
        const float4 e = *reinterpret_cast<const float4*>(recvh + (buf * 16 + (lane & 15)) * 4);
        ns.hi = e.x; ns.lo = e.y; hxs = e.z; hys = e.w;
      }
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) {
        const float h = __shfl_xor_sync(0xffffffffu, ns.hi, o), l = __shfl_xor_sync(0xffffffffu, ns.lo, o);
        ns.add_nr(h, l);
        hxs += __shfl_xor_sync(0xffffffffu, hxs, o);
        hys += __shfl_xor_sync(0xffffffffu, hys, o);
      }
      T beta, tr, ti, sr, si;
      reflector_rf(ns.value(), alpha.x, alpha.y, beta, tr, ti, sr, si);
      if (lane == 0 && rank == 0 && !(isfinite(beta) && isfinite(sr) && isfinite(si)))
        atomicOr(a.err, DEVERR_NUMERIC);
      const cx<T> sc = mk<T>(sr, si), tau = mk<T>(tr, ti);
      if (!mbar_wait_cl(&sh.mb[buf], (uint32_t)((jn >> 1) & 1))) ok = false;
      cx<T> S;
      {
        const unsigned char* base = sh.recvm + buf * 16 * MSGS + col * sizeof(cx<T>);
        cx<T> v[16];
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = r < CS ? *reinterpret_cast<const cx<T>*>(base + r * MSGS) : zero;
#pragma unroll
        for (int h = 8; h > 0; h >>= 1)
#pragma unroll
          for (int r = 0; r < h; ++r) v[r] = cadd<T>(v[r], v[r + h]);
        S = v[0];
      }
      if (jp >= 0) S = csub<T>(S, cmul<T>(mk<T>(hxs, hys), cws));
      const bool u = lane > jn && lane < kb;
      const cx<T> cwl = u ? cmul<T>(cconj<T>(tau), cadd<T>(pc, cmul<T>(cconj<T>(sc), S))) : zero;
      if (lane < jn) {
        const cx<T> gv = cmul<T>(cconj<T>(scl_l), cadd<T>(cconj<T>(pc), cmul<T>(sc, cconj<T>(S))));
        sh.Ts[lane * (KBMAX + 1) + jn] = gv;
      }
      cx<T>* bb = sh.bc + buf * (SLOTS + 2);
      bb[lane] = cwl;
      if (lane == 0) { bb[SLOTS] = sc; sh.taus[jn] = tau; sh.scl[jn] = sc; sh.bet[jn] = mk<T>(beta, 0); }
    }
    asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory");
    {
      const cx<T>* bb = sh.bc + buf * (SLOTS + 2);
      cw = bb[lane];
      cws = cmul_rn(bb[SLOTS], cw);
      // the next pivot column's pair, read directly (bit-identical to its lane's cws)
      cwj = bb[min(jn + 1, SLOTS - 1)];
      cwsj = cmul_rn(bb[SLOTS], cwj);
    }
  }
  if (!ok && tid == 0) atomicOr(a.err, DEVERR_TIMEOUT);
  __syncthreads();

  if (rank == CS - 1) panel_t_factor<T, NW>(sh, kb, a);
  // ---- V (v = scale * raw column below the pivot, unit diagonal) and R / zeros into A:
  //      the top rows from rank 0's shared memory, the slab from registers
  if (lane < kb) {
    const cx<T> sc = sh.scl[lane], be = sh.bet[lane];
    if (rank == 0 && rw >= 0)
      for (int t = rw; t < kb; t += RW) {
        const cx<T> pv = Pt[t * ldp + lane];
        a.V[(k0 + t) * a.ldv + k0 + lane] = (t == lane) ? mk<T>(1, 0) : (t > lane ? cmul<T>(sc, pv) : zero);
        a.A[(k0 + t) * a.lda + k0 + lane] = (lane > t) ? pv : (lane == t ? be : zero);
      }
    cx<T>* vd = a.V + (k0 + s0 + q0) * a.ldv + k0 + lane;
    cx<T>* ad = a.A + (k0 + s0 + q0) * a.lda + k0 + lane;
#pragma unroll
    for (int r = 0; r < RPW; ++r)
      if (r < cnt) { vd[r * a.ldv] = cmul<T>(sc, R[r]); ad[r * a.lda] = zero; }
  }
  cl.sync();
}

template <typename T>
__global__ void k_eye(cx<T>* Q, long long ldq, int m, int n) {
  pdl_launch_dependents();
  pdl_wait();
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)m * n) return;
  int i = (int)(idx / n), j = (int)(idx % n);
  Q[i * ldq + j] = mk<T>(i == j ? T(1) : T(0), 0);
}

// Q[i][i] += 1 for i < n (the identity of Q = [I; 0] - V W added after the GEMM)
template <typename T>
__global__ void k_add_eye(cx<T>* Q, long long ldq, int n) {
  pdl_launch_dependents();
  pdl_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) Q[i * ldq + i].x += T(1);
}

template <typename T> __device__ __forceinline__ void cp_async_cx(cx<T>* dst_smem, const cx<T>* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst_smem)),
               "l"(src), "n"((int)sizeof(cx<T>)) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// ------------------------------------------------------ outer compact-WY factor
// T of an outer block straight from its Householder scalars and the Gram matrix
// G = V^dag V of the block: with U the strict upper part of G, T^{-1} = diag(1/tau) + U,
// so column j of T solves t_i = tau_i (delta_ij - sum_{k > i} U_ik t_k), i = j, ..., 0 (a
// form that also covers tau_i = 0, H_i = I). The columns are independent: one warp per
// column, lane = row (rows lane + 32 q); step k finalises t_k on its lane and broadcasts
// it, and the rows above take U_ik t_k, with U_ik = conj(G[k, i]) read along row k of G.
constexpr int TB_NT = 256;
// complex64 stages the rows of G the CTA's columns read into shared memory (at most
// NBO x NBO x 8 bytes = 128 KB); complex128 reads G in place
template <typename T> constexpr bool kTbStage = sizeof(cx<T>) == 8;
template <typename T> size_t t_cols_smem(int kbo, int cta) {
  const int rows = std::min(kbo, (cta + 1) * (TB_NT / 32));
  return kTbStage<T> ? (size_t)rows * kbo * sizeof(cx<T>) : 0;
}
template <typename T>
__global__ void __launch_bounds__(TB_NT) k_t_cols(cx<T>* Tb, int ldt, const cx<T>* __restrict__ G, int ldg,
                                                   const cx<T>* __restrict__ tau, int kbo) {
  extern __shared__ __align__(16) unsigned char sm[];
  pdl_launch_dependents();
  pdl_wait();
  constexpr int Q = NBO / 32;  // rows per lane
  const int lane = threadIdx.x & 31;
  const int j = blockIdx.x * (TB_NT / 32) + (threadIdx.x >> 5);
  const int rows = min(kbo, (int)(blockIdx.x + 1) * (TB_NT / 32));  // rows of G this CTA reads
  const cx<T>* Gr = G;
  int ldr = ldg;
  if constexpr (kTbStage<T>) {
    cx<T>* Gs = reinterpret_cast<cx<T>*>(sm);
    for (int o = threadIdx.x; o < rows * kbo; o += TB_NT)
      cp_async_cx<T>(Gs + o, G + (long long)(o / kbo) * ldg + o % kbo);
    cp_async_wait_all();
    __syncthreads();
    Gr = Gs; ldr = kbo;
  }
  if (j >= kbo) return;
  const cx<T> zero = mk<T>(0, 0);
  cx<T> acc[Q], t[Q], tl[Q], g[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int i = lane + 32 * q;
    acc[q] = zero; t[q] = zero;
    tl[q] = i < kbo ? tau[i] : zero;
    g[q] = (i < j) ? Gr[(long long)j * ldr + i] : zero;  // row j, for the first step
  }
  for (int k = j; k >= 0; --k) {
    const int qk = k >> 5, lk = k & 31;
    // row k - 1 of G for the next step, loaded ahead of this step's arithmetic
    cx<T> gn[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int i = lane + 32 * q;
      gn[q] = (k > 0 && i < k - 1) ? Gr[(long long)(k - 1) * ldr + i] : zero;
    }
    cx<T> ak = acc[0], tk_l = tl[0];
#pragma unroll
    for (int q = 1; q < Q; ++q)
      if (qk == q) { ak = acc[q]; tk_l = tl[q]; }
    const cx<T> tk = shfl_cx<T>(cmul<T>(tk_l, csub<T>(mk<T>(k == j ? T(1) : T(0), T(0)), ak)), lk);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      if (qk == q && lane == lk) t[q] = tk;
      cfma<T>(acc[q], cconj<T>(g[q]), tk);  // g = 0 on rows i >= k
      g[q] = gn[q];
    }
  }
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int i = lane + 32 * q;
    if (i < kbo) Tb[(long long)i * ldt + j] = t[q];  // t = 0 below the diagonal
  }
}
template <typename T> bool g_tc_attr = false;

// Blocked form for inner panels of 32 columns: the inner factors T_bb that the panels left on
// the diagonal of Tb are the inverses of the diagonal blocks of D + U, so column j of T is
// solved block by block, b = block(j), ..., 0:
//   t_b = T_bb (e_j[b] - acc_b),   acc_a += U_ab t_b for a < b,
// U_ab[i][k] = G[32a + i][32b + k] = conj(G[32b + k][32a + i]). The tau_i = 0 rows come
// out zero as in the column form, since those rows of T_bb are zero. One warp per column,
// lane = row within a block; the vectors a step broadcasts go through a per-warp buffer.
constexpr int TBB = 32;
template <typename T> size_t t_block_smem(int kbo) {
  const int nbk = (int)ceil_div(kbo, TBB), ur = TBB * (nbk - 1);
  return ((size_t)ur * ur + (size_t)TBB * nbk * (TBB + 1) + (size_t)(TB_NT / 32) * TBB) * sizeof(cx<T>);
}
template <typename T>
__global__ void __launch_bounds__(TB_NT) k_t_block(cx<T>* Tb, int ldt, const cx<T>* __restrict__ G, int ldg,
                                                   int kbo) {
  extern __shared__ __align__(16) unsigned char sm[];
  pdl_launch_dependents();
  pdl_wait();
  constexpr int Q = NBO / TBB, LDD = TBB + 1;
  const int nbk = (int)ceil_div(kbo, TBB), ur = TBB * (nbk - 1);
  cx<T>* Us = reinterpret_cast<cx<T>*>(sm);  // G[32 + r][c], r, c < ur (rows past kbo zero)
  cx<T>* Dg = Us + (size_t)ur * ur;          // the diagonal blocks of T, row i: T[i][32 block(i) + k]
  cx<T>* wb = Dg + (size_t)TBB * nbk * LDD;  // per warp: the vector being broadcast
  const cx<T> zero = mk<T>(0, 0);
  // staged with cp.async (no load waits on its store), zeros stored directly
  for (int o = threadIdx.x; o < ur * ur; o += TB_NT) {
    const int r = o / ur, c = o % ur;
    if (TBB + r < kbo) cp_async_cx<T>(Us + o, G + (long long)(TBB + r) * ldg + c);
    else Us[o] = zero;
  }
  for (int o = threadIdx.x; o < TBB * nbk * TBB; o += TB_NT) {
    const int i = o / TBB, k = o % TBB, c = (i / TBB) * TBB + k;
    if (i < kbo && c < kbo) cp_async_cx<T>(Dg + i * LDD + k, Tb + (long long)i * ldt + c);
    else Dg[i * LDD + k] = zero;
  }
  cp_async_wait_all();
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = blockIdx.x * (TB_NT / 32) + warp;
  if (j >= kbo) return;
  cx<T>* w = wb + warp * TBB;
  const int qj = j / TBB, jl = j % TBB;
  cx<T> acc[Q], t[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) { acc[q] = zero; t[q] = zero; }
  for (int b = qj; b >= 0; --b) {
    cx<T> r = zero;
#pragma unroll
    for (int q = 0; q < Q; ++q)
      if (q == b) r = csub<T>(mk<T>(b == qj && lane == jl ? T(1) : T(0), T(0)), acc[q]);
    w[lane] = r;
    __syncwarp();
    // t_b = T_bb r (upper triangular: the zeros below its diagonal are stored)
    cx<T> s0 = zero, s1 = zero;
    const cx<T>* drow = Dg + (TBB * b + lane) * LDD;
#pragma unroll
    for (int k = 0; k < TBB; k += 2) {
      cfma<T>(s0, drow[k], w[k]);
      cfma<T>(s1, drow[k + 1], w[k + 1]);
    }
    const cx<T> tb = cadd<T>(s0, s1);
    __syncwarp();
#pragma unroll
    for (int q = 0; q < Q; ++q)
      if (q == b) t[q] = tb;
    if (b == 0) break;
    w[lane] = tb;
    __syncwarp();
    // acc_a += U_ab t_b for the blocks a < b
    const cx<T>* urow = Us + (size_t)(TBB * b - TBB) * ur;
#pragma unroll
    for (int a = 0; a < Q - 1; ++a) {
      if (a < b) {
        cx<T> u0 = zero, u1 = zero;
#pragma unroll
        for (int k = 0; k < TBB; k += 2) {
          cfma<T>(u0, cconj<T>(urow[(size_t)k * ur + TBB * a + lane]), w[k]);
          cfma<T>(u1, cconj<T>(urow[(size_t)(k + 1) * ur + TBB * a + lane]), w[k + 1]);
        }
        acc[a] = cadd<T>(acc[a], cadd<T>(u0, u1));
      }
    }
    __syncwarp();
  }
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int i = TBB * q + lane;
    if (i < kbo) Tb[(long long)i * ldt + j] = t[q];  // t = 0 below the diagonal
  }
}
template <typename T> bool g_tb_attr = false;

// ------------------------------------------------------ fused narrow block-reflector update
// C <- (I - V T V^dag)^dag C = C - V T^dag (V^dag C) for the columns of an outer block right
// of a panel: kb <= 32 reflectors, nc <= WY_NC columns, C and V of mr rows. One cooperative
// launch, each CTA a slab of rpb rows held in shared memory:
//   (1) partial V^dag C over the slab; (2) the partials summed, one output per lane;
//   (3) W2 = T^dag W, then C -= V W2 on the slab.
// Grid barriers separate the phases; their waits are bounded (DEVERR_TIMEOUT) and the
// cooperative launch guarantees that every CTA is resident.
constexpr int WY_NT = 256;
constexpr int WY_NC = 128;
constexpr int WY_KB = 32;
constexpr int WY_PW = 19;  // partials a warp sums in phase (2): CTAs <= 8 x 19 = 152


template <typename T, int NQ>  // NQ = ceil(nc / 32) column groups of 32 (nc <= WY_NC)
__global__ void __launch_bounds__(WY_NT) k_apply_wy(cx<T>* C, long long ldc, const cx<T>* V,
                                                    long long ldv, const cx<T>* Tt, int ldt, int mr,
                                                    int nc, int kb, int rpb, cx<T>* part, cx<T>* Wg,
                                                    unsigned* bar, unsigned* err) {
  extern __shared__ __align__(16) unsigned char sm[];
  cx<T>* Vs = reinterpret_cast<cx<T>*>(sm);  // rpb x kb
  cx<T>* Cs = Vs + (size_t)rpb * kb;         // rpb x nc
  cx<T>* Ws = Cs + (size_t)rpb * nc;         // kb x nc
  cx<T>* Ts = Ws + (size_t)kb * nc;          // kb x kb
  const int tid = threadIdx.x;
  const unsigned G = gridDim.x;
  const int b = blockIdx.x;
  const int r0 = b * rpb, nr = max(0, min(rpb, mr - r0));
  const cx<T> zero = mk<T>(0, 0);
  for (int i = tid; i < nr * kb; i += WY_NT) cp_async_cx<T>(Vs + i, V + (long long)(r0 + i / kb) * ldv + i % kb);
  for (int i = tid; i < nr * nc; i += WY_NT) cp_async_cx<T>(Cs + i, C + (long long)(r0 + i / nc) * ldc + i % nc);
  for (int i = tid; i < kb * kb; i += WY_NT) cp_async_cx<T>(Ts + i, Tt + (long long)(i / kb) * ldt + i % kb);
  cp_async_wait_all();
  __syncthreads();
  // register tiles: columns c_q = lane + 32 q (q < 4), and reflectors a_p (phase 1, 3a)
  // or rows r_p (phase 3b) = warp + 8 p; 16 independent accumulators per thread
  const int lane = tid & 31, wg = tid >> 5;
  constexpr int NP = WY_KB / 8;
  // (1) partial V^dag C
  {
    cx<T> acc[NP][NQ];
#pragma unroll
    for (int p = 0; p < NP; ++p)
#pragma unroll
      for (int q = 0; q < NQ; ++q) acc[p][q] = zero;
#pragma unroll 2
    for (int r = 0; r < nr; ++r) {
      cx<T> x[NQ], v[NP];
#pragma unroll
      for (int q = 0; q < NQ; ++q) x[q] = (lane + 32 * q < nc) ? Cs[r * nc + lane + 32 * q] : zero;
#pragma unroll
      for (int p = 0; p < NP; ++p) v[p] = (wg + 8 * p < kb) ? cconj<T>(Vs[r * kb + wg + 8 * p]) : zero;
#pragma unroll
      for (int p = 0; p < NP; ++p)
#pragma unroll
        for (int q = 0; q < NQ; ++q) cfma<T>(acc[p][q], v[p], x[q]);
    }
    // through shared memory (Ws is free until phase 3) so that the CTA's partial block,
    // stored [CTA][column][a], is written with coalesced stores
#pragma unroll
    for (int p = 0; p < NP; ++p)
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const int aa = wg + 8 * p, c = lane + 32 * q;
        if (aa < kb && c < nc) Ws[c * kb + aa] = acc[p][q];
      }
    __syncthreads();
    for (int i = tid; i < kb * nc; i += WY_NT) part[(size_t)b * kb * nc + i] = Ws[i];
  }
  if (!grid_barrier(bar, G, err)) return;
  // (2) one CTA per column c: lane = reflector index a, the warps split the G partials
  //     of W[:, c] = V^dag C[:, c] (stored [CTA][column][a], so a warp reads 32 consecutive
  //     values; each warp's share of the partials is loaded at once, then summed as a tree);
  //     warp 0 sums the warps' values and applies T^dag, so W2 = T^dag W is formed once
  {
    __shared__ cx<T> red[WY_NT / 32][32];
    __shared__ cx<T> wsum[32];
    const int warp = tid >> 5, lane2 = tid & 31;
    constexpr unsigned WS = WY_NT / 32;
    for (int c = b; c < nc; c += (int)G) {
      cx<T> acc = zero;
      if (lane2 < kb) {
        const size_t off = (size_t)c * kb + lane2, stride = (size_t)kb * nc;
        cx<T> v[WY_PW];
#pragma unroll
        for (int i = 0; i < WY_PW; ++i) {
          const unsigned z = warp + WS * i;
          v[i] = z < G ? part[z * stride + off] : zero;
        }
#pragma unroll
        for (int h = 16; h > 0; h >>= 1)
#pragma unroll
          for (int i = 0; i < h; ++i)
            if (i + h < WY_PW) v[i] = cadd<T>(v[i], v[i + h]);
        acc = v[0];
      }
      red[warp][lane2] = acc;
      __syncthreads();
      if (warp == 0) {
        cx<T> wv = zero;
        for (int w = 0; w < (int)WS; ++w) wv = cadd<T>(wv, red[w][lane2]);
        wsum[lane2] = wv;
        __syncwarp();
        // W2[a] = sum_k conj(T[k][a]) W[k] (T upper triangular: its zeros are stored)
        cx<T> a0 = zero, a1 = zero;
        if (lane2 < kb) {
          for (int k = 0; k + 1 < kb; k += 2) {
            cfma<T>(a0, cconj<T>(Ts[k * kb + lane2]), wsum[k]);
            cfma<T>(a1, cconj<T>(Ts[(k + 1) * kb + lane2]), wsum[k + 1]);
          }
          if (kb & 1) cfma<T>(a0, cconj<T>(Ts[(kb - 1) * kb + lane2]), wsum[kb - 1]);
          Wg[(size_t)lane2 * nc + c] = cadd<T>(a0, a1);
        }
      }
      __syncthreads();
    }
  }
  if (!grid_barrier(bar, G, err)) return;
  // (3) W2 into shared memory, then C -= V W2 on the slab
  for (int i = tid; i < kb * nc; i += WY_NT) cp_async_cx<T>(Ws + i, Wg + i);
  cp_async_wait_all();
  __syncthreads();
  // (3b) C -= V W2 on the slab: 32-row tiles (rows r0c + warp + 8 p), then 8-row steps
  int r0c = 0;
  for (; r0c + 8 * NP <= nr; r0c += 8 * NP) {
    cx<T> acc[NP][NQ];
#pragma unroll
    for (int p = 0; p < NP; ++p)
#pragma unroll
      for (int q = 0; q < NQ; ++q) acc[p][q] = zero;
    for (int k = 0; k < kb; ++k) {
      cx<T> w[NQ], v[NP];
#pragma unroll
      for (int q = 0; q < NQ; ++q) w[q] = (lane + 32 * q < nc) ? Ws[k * nc + lane + 32 * q] : zero;
#pragma unroll
      for (int p = 0; p < NP; ++p) v[p] = Vs[(r0c + wg + 8 * p) * kb + k];
#pragma unroll
      for (int p = 0; p < NP; ++p)
#pragma unroll
        for (int q = 0; q < NQ; ++q) cfma<T>(acc[p][q], v[p], w[q]);
    }
#pragma unroll
    for (int p = 0; p < NP; ++p)
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const int r = r0c + wg + 8 * p, c = lane + 32 * q;
        if (c < nc) C[(long long)(r0 + r) * ldc + c] = csub<T>(Cs[r * nc + c], acc[p][q]);
      }
  }
  for (; r0c < nr; r0c += 8) {
    const int r = r0c + wg;
    cx<T> acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] = zero;
    if (r < nr) {
      for (int k = 0; k < kb; ++k) {
        const cx<T> v = Vs[r * kb + k];
#pragma unroll
        for (int q = 0; q < NQ; ++q)
          if (lane + 32 * q < nc) cfma<T>(acc[q], v, Ws[k * nc + lane + 32 * q]);
      }
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const int c = lane + 32 * q;
        if (c < nc) C[(long long)(r0 + r) * ldc + c] = csub<T>(Cs[r * nc + c], acc[q]);
      }
    }
  }
}

int g_nsm = 0;
int num_sms() {
  if (g_nsm == 0) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
      g_nsm = v;
    else
      g_nsm = 148;
  }
  return g_nsm;
}

thread_local int g_concurrency = 1;  // see ConcurrencyScope

template <typename T> size_t wy_smem(int rpb, int kb, int nc) {
  return ((size_t)rpb * kb + (size_t)rpb * nc + (size_t)kb * nc + (size_t)kb * kb) * sizeof(cx<T>);
}

// Rows per CTA of the fused update: one CTA per SM at most (co-residency of a
// cooperative launch), at least 8 rows per CTA; beside other bond updates at most
// num_sms / min(n, 4) CTAs (ConcurrencyScope).
template <typename T> int wy_rows_per_block(int mr, int kb, int nc) {
  if (kb < 1 || kb > WY_KB || nc < 1 || nc > WY_NC || mr < 1) return 0;
  const size_t smax = (size_t)48 * 1024 * 4;
  const int sms = num_sms();
  const int full = std::max(8, (int)ceil_div(mr, std::min(sms, (WY_NT / 32) * WY_PW)));
  if (g_concurrency > 1) {
    const int cap = std::max(1, sms / std::min(g_concurrency, 4));
    const int rpb = std::max(8, (int)ceil_div(mr, std::min(cap, (WY_NT / 32) * WY_PW)));
    if (wy_smem<T>(rpb, kb, nc) <= smax) return rpb;
  }
  return wy_smem<T>(full, kb, nc) <= smax ? full : 0;
}

template <typename T> bool g_wy_attr = false;

template <typename T>
int apply_wy(cx<T>* C, long long ldc, const cx<T>* V, long long ldv, const cx<T>* Tt, int ldt, int mr,
             int nc, int kb, int rpb, const QrScratch<T>& s, cudaStream_t st, unsigned* err) {
  const int G = (int)ceil_div(mr, rpb);
  const size_t smem = wy_smem<T>(rpb, kb, nc);
  // the partial sums hold one block per CTA, for at most one CTA per SM
  if (G > std::max(num_sms(), 1) || G > (WY_NT / 32) * WY_PW) {
    set_last_message("QR narrow update: more CTAs than its partial-sum buffer holds");
    return QRTEBD_ERR_INVALID_ARG;
  }
  if (!g_wy_attr<T>) {
    QR_CUDA_TRY(cudaFuncSetAttribute(k_apply_wy<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 48 * 1024 * 4));
    QR_CUDA_TRY(cudaFuncSetAttribute(k_apply_wy<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 48 * 1024 * 4));
    QR_CUDA_TRY(cudaFuncSetAttribute(k_apply_wy<T, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 48 * 1024 * 4));
    QR_CUDA_TRY(cudaFuncSetAttribute(k_apply_wy<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 48 * 1024 * 4));
    g_wy_attr<T> = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)G, 1, 1);
  cfg.blockDim = dim3(WY_NT, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at; cfg.numAttrs = 1;
  ProfScope prof(PROF_SIMT_GEMM, st, 16.0 * mr * nc * kb);
  // register tiles only as wide as the columns: ceil(nc / 32) groups of 32
  switch ((nc + 31) / 32) {
    case 1: QR_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_apply_wy<T, 1>, C, ldc, V, ldv, Tt, ldt, mr, nc, kb, rpb,
                                           s.wy_part, s.wy_W, s.bar, err)); break;
    case 2: QR_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_apply_wy<T, 2>, C, ldc, V, ldv, Tt, ldt, mr, nc, kb, rpb,
                                           s.wy_part, s.wy_W, s.bar, err)); break;
    case 3: QR_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_apply_wy<T, 3>, C, ldc, V, ldv, Tt, ldt, mr, nc, kb, rpb,
                                           s.wy_part, s.wy_W, s.bar, err)); break;
    default: QR_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_apply_wy<T, 4>, C, ldc, V, ldv, Tt, ldt, mr, nc, kb, rpb,
                                            s.wy_part, s.wy_W, s.bar, err)); break;
  }
  note_launch();
  return QRTEBD_OK;
}

struct ClusterChoice { int cs; int rps; int kb; };


// Largest cluster the device co-schedules for the panel kernel (16 needs the
// non-portable opt-in; probed once per process, falls back to 8), and the opt-in
// dynamic shared memory per block.
int g_max_cluster = 0;
int g_smem_cap = 0;

int smem_cap() {
  if (g_smem_cap == 0) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess && v > 0)
      g_smem_cap = v;
    else
      g_smem_cap = 227 * 1024;
  }
  return g_smem_cap;
}

// Cluster size, slab rows per CTA and panel width for a panel of mr rows: the
// smallest power-of-two cluster giving every CTA at most ~320 slab rows for complex64 (a
// 5120-row panel takes 16 CTAs, a 2048-row one 8, which leaves SMs to concurrent updates;
// the panel is bound by the latency of its per-column exchange), at most ~24 for
// complex128, whose panel is bound by the FP64 work of each CTA (~230 cycles per row and
// column on B300's FP64 pipe, against ~3k for a column's exchange and reflector), grown
// (then the width halved) until the panel fits in shared memory.
template <typename T> ClusterChoice choose_cluster(int mr, int kb_want) {
  const int cmax = g_max_cluster > 0 ? g_max_cluster : 16;
  const size_t cap = (size_t)smem_cap();
  const int rows = std::is_same<T, double>::value ? 24 : 320;
  int cs = 1;
  while (cs < cmax && (long long)cs * rows < mr) cs *= 2;
  for (int kb = kb_want; kb >= 1; kb /= 2) {
    for (int s = cs; s <= cmax; s *= 2) {
      const int rps = (int)ceil_div(std::max(mr - kb, 0), s);
      if (panel_smem_bytes<T>(rps, kb) <= cap) return ClusterChoice{s, rps, kb};
    }
  }
  return ClusterChoice{-1, 0, kb_want};
}

// Complex128 panels whose 16-CTA cluster would hold more than ~24 slab rows a CTA run in the
// grid form on G <= 148 CTAs of ~40 slab rows (a 5120-row panel: 128 CTAs of 40 rows,
// against 16 of 320 in the cluster form).
constexpr int PG_ROWS = 40;
template <typename T> bool pg_shape(int mr, int kb, int* G, int* rps) {
  if (!std::is_same<T, double>::value) return false;
  const int S = mr - kb;
  if (S <= 16 * 24) return false;
  const int g = (int)std::min<long long>(std::min(PG_MAX, std::max(num_sms(), 1)), ceil_div(S, PG_ROWS));
  *G = g;
  *rps = (int)ceil_div(S, g);
  return true;
}
template <typename T> size_t g_pg_attr = 0;  // dynamic shared memory the attribute allows

template <typename T> int launch_panel_g(const PanelArgs<T>& pa, int G, const QrScratch<T>& s, cudaStream_t st) {
  const size_t smem = panel_smem_bytes<T>(pa.rps, pa.kb);
  const int mr = pa.m - pa.k0;
  // the grid barrier's flag takes a little static shared memory: keep 1 KB of the opt-in size
  if (pa.kb < 1 || pa.kb > KBMAX || mr < pa.kb || G < 1 || G > PG_MAX || (long long)pa.rps * G < mr - pa.kb ||
      smem > (size_t)smem_cap() - 1024 || !s.pg) {
    set_last_message("QR grid panel: invalid shape");
    return QRTEBD_ERR_INVALID_ARG;
  }
  if (g_pg_attr<T> < smem) {
    QR_CUDA_TRY(cudaFuncSetAttribute(k_qr_panel_g<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    g_pg_attr<T> = smem;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)G, 1, 1);
  cfg.blockDim = dim3(PT, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at; cfg.numAttrs = 1;
  ProfScope prof(PROF_QR_PANEL, st, 8.0 * mr * pa.kb * pa.kb, 3.0 * mr * pa.kb * sizeof(cx<T>));
  QR_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_qr_panel_g<T>, pa, s.pg, s.bar + 16));
  note_launch();
  return QRTEBD_OK;
}

template <typename T> bool g_attr_done = false;

template <typename T> int set_panel_attrs() {
  if (g_attr_done<T>) return QRTEBD_OK;
  QR_CUDA_TRY(cudaFuncSetAttribute(k_qr_panel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_cap()));
  QR_CUDA_TRY(cudaFuncSetAttribute(k_qr_panel<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  if constexpr (std::is_same<T, float>::value) {
    QR_CUDA_TRY(cudaFuncSetAttribute(k_qr_panel_rf<RF_RPW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     smem_cap()));
    QR_CUDA_TRY(cudaFuncSetAttribute(k_qr_panel_rf<RF_RPW>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  }
  g_attr_done<T> = true;
  return QRTEBD_OK;
}

// Probe once whether 16-CTA clusters of the panel kernel (at the largest shared
// memory size) can be co-scheduled; otherwise cap clusters at 8 CTAs.
template <typename T> int probe_max_cluster() {
  if (g_max_cluster > 0) return QRTEBD_OK;
  QR_TRY(set_panel_attrs<T>());
  cudaLaunchConfig_t q = {};
  q.gridDim = dim3(16, 1, 1); q.blockDim = dim3(PT, 1, 1); q.dynamicSmemBytes = smem_cap();
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
  // the register-file form whenever each warp's slab share fits (complex64)
  const bool rf = std::is_same<T, float>::value && pa.rps <= (RF_NT / 32 - 1) * RF_RPW;
  const size_t smem = rf ? panel_rf_smem_bytes<T>(pa.kb) : panel_smem_bytes<T>(pa.rps, pa.kb);
  const int mr = pa.m - pa.k0;
  if (pa.kb < 1 || pa.kb > KBMAX || mr < pa.kb || cs < 1 || cs > 16 || pa.rps < 0 ||
      (long long)pa.rps * cs < mr - pa.kb || smem > (size_t)smem_cap()) {
    set_last_message("QR panel: invalid cluster shape");
    return QRTEBD_ERR_INVALID_ARG;
  }
  QR_TRY(set_panel_attrs<T>());
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cs, 1, 1);
  cfg.blockDim = dim3(rf ? RF_NT : PT, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs; attr[0].val.clusterDim.y = 1; attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr; cfg.numAttrs = 2;
  // algorithmic work of a Householder panel: 8 mr kb^2 real flops; traffic: the panel
  // read once, V and R/zeros written once
  ProfScope prof(PROF_QR_PANEL, st, 8.0 * mr * pa.kb * pa.kb, 3.0 * mr * pa.kb * sizeof(cx<T>));
  if constexpr (std::is_same<T, float>::value) {
    if (rf) QR_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_qr_panel_rf<RF_RPW>, pa));
    else QR_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_qr_panel<T>, pa));
  } else {
    QR_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_qr_panel<T>, pa));
  }
  note_launch();
  return QRTEBD_OK;
}

// Side streams for look-ahead, one per (device, main stream), with reusable events.
struct SideStream {
  cudaStream_t st = nullptr;  // the look-ahead work, least priority
  cudaStream_t hp = nullptr;  // the panel chain, greatest priority (forked from the caller's)
  std::vector<cudaEvent_t> ev;
};
std::mutex g_side_mu;
std::map<std::pair<int, cudaStream_t>, SideStream> g_side;

int side_stream(cudaStream_t main, int nev, SideStream** out) {
  int dev = 0;
  QR_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_side_mu);
  SideStream& ss = g_side[std::make_pair(dev, main)];
  if (!ss.st) {
    // the look-ahead work at the least priority, the panel chain at the greatest, so that
    // freed SMs go to the chain whenever both have blocks waiting (the caller's stream
    // itself may have the least priority)
    int lo = 0, hi = 0;
    QR_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    QR_CUDA_TRY(cudaStreamCreateWithPriority(&ss.st, cudaStreamNonBlocking, lo));
    QR_CUDA_TRY(cudaStreamCreateWithPriority(&ss.hp, cudaStreamNonBlocking, hi));
  }
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

ConcurrencyScope::ConcurrencyScope(int n) : prev_(g_concurrency) { g_concurrency = std::max(1, n); }
ConcurrencyScope::~ConcurrencyScope() { g_concurrency = prev_; }
int concurrency() { return g_concurrency; }

int qr_panel_width(int m, int n, int elem_bytes) {
  int kb = n < KBMAX ? n : KBMAX;
  if (kb < 1) kb = 1;
  if (elem_bytes == 16) {
    // a complex128 panel in the grid form holds ~40 slab rows a CTA: the full width fits
    int G = 0, rps = 0;
    if (pg_shape<double>(m, kb, &G, &rps) && panel_smem_bytes<double>(rps, kb) <= (size_t)smem_cap() - 1024)
      return kb;
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
  s.VT = ar.take<cx<T>>((size_t)m * n);
  s.Tf = ar.take<cx<T>>((size_t)(n + nbo) * nbo);
  s.W = ar.take<cx<T>>((size_t)nbo * n);
  s.W2 = ar.take<cx<T>>((size_t)nbo * n);
  s.W2s = ar.take<cx<T>>((size_t)nbo * n);
  if (std::is_same<T, float>::value) {
    s.Tall = ar.take<cx<T>>((size_t)n * n);
    s.Cb = ar.take<cx<T>>((size_t)n * nbo);
    s.Xb = ar.take<cx<T>>((size_t)n * nbo);
    s.Wq = ar.take<cx<T>>((size_t)n * n);
  }
  s.G = ar.take<cx<T>>((size_t)nbo * nbo);
  s.wy_part = ar.take<cx<T>>((size_t)std::max(num_sms(), 1) * WY_KB * WY_NC);
  s.wy_W = ar.take<cx<T>>((size_t)WY_KB * WY_NC);
  if (std::is_same<T, double>::value) s.pg = ar.take<cx<T>>((size_t)2 * PG_MAX * (SLOTS + 1));
  s.bar = ar.take<unsigned>(64);
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
                   QrScratch<T>& s, cudaStream_t st_in, unsigned* err, const QrGemm<T>* gm,
                   const QrGemm<T>* side) {
  cudaStream_t st = st_in;  // the panel chain; with look-ahead, a greatest-priority fork
  if (m < n || n < 1) return QRTEBD_ERR_INVALID_ARG;
  QR_TRY(probe_max_cluster<T>());
  const int nb = qr_panel_width(m, n, sizeof(cx<T>));
  if (nb < 1) { set_last_message("QR: matrix too tall for the shared-memory panel"); return QRTEBD_ERR_INVALID_ARG; }
  const long long ldv = n;
  const int nbo = NBO;  // outer block: inner panels of nb columns inside it
  const cx<T> one = mk<T>(1, 0), zero = mk<T>(0, 0), mone = mk<T>(-1, 0);
  const int nblk = (int)ceil_div(n, nbo);
  SideStream* ss = nullptr;
  if (side && side->fn && nblk > 2) {
    QR_TRY(side_stream(st_in, 3 * nblk + 3, &ss));
    QR_CUDA_TRY(cudaEventRecord(ss->ev[2 * nblk], st_in));
    QR_CUDA_TRY(cudaStreamWaitEvent(ss->hp, ss->ev[2 * nblk], 0));
    st = ss->hp;
  }
  // V must be zero above each panel's diagonal block: an outer block reads the rows
  // above its later inner panels, which those panels do not write
  QR_CUDA_TRY(cudaMemsetAsync(s.V, 0, (size_t)m * n * sizeof(cx<T>), st));
  QR_CUDA_TRY(cudaMemsetAsync(s.bar, 0, 32 * sizeof(unsigned), st));  // [0..1] narrow update, [16..17] grid panel
  // complex64 with look-ahead: the compact-WY factor of the whole QR is assembled on the side
  // stream block by block, and the explicit Q then takes two GEMMs,
  // Q = [I; 0] - V (T_all V_top^dag), instead of one backward step per outer block
  const bool qfast = std::is_same<T, float>::value && ss != nullptr && s.Tall != nullptr;
  if (qfast) QR_CUDA_TRY(cudaMemsetAsync(s.Tall, 0, (size_t)n * n * sizeof(cx<T>), st));
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
      if (cc.cs < 0 || cc.kb != kb) { cc.kb = kb; cc.cs = 16; cc.rps = (int)ceil_div(mr - kb, 16); }
      cx<T>* Ti = Tb + (size_t)(ki - ko) * nbo + (ki - ko);
      PanelArgs<T> pa{A, lda, m, ki, kb, s.V, ldv, s.tau, Ti, nbo, cc.rps, err};
      int pgG = 0, pgR = 0;
      bool grid_form = false;
      if constexpr (std::is_same<T, double>::value) grid_form = pg_shape<T>(mr, kb, &pgG, &pgR) && s.pg;
      if (grid_form) {
        if constexpr (std::is_same<T, double>::value) {
          PanelArgs<T> p2 = pa;
          p2.rps = pgR;
          QR_TRY(launch_panel_g<T>(p2, pgG, s, st));
        }
      } else {
        QR_TRY(launch_panel<T>(pa, cc.cs, st));
      }
      // inner update: the rest of this outer block
      const int nc = ko + kbo - ki - kb;
      const int rpb = nc > 0 ? wy_rows_per_block<T>(mr, kb, nc) : 0;
      if (rpb > 0) {
        QR_TRY(apply_wy<T>(A + (long long)ki * lda + ki + kb, lda, s.V + (long long)ki * ldv + ki, ldv,
                           Ti, nbo, mr, nc, kb, rpb, s, st, err));
      } else if (nc > 0) {
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
    cx<T>* VTb = s.VT + (long long)ko * ldv + ko;
    const int nc = n - ko - kbo;
    const int n1 = ss ? std::min(nbo, nc) : nc;
    // T of the outer block from G = V^dag V (leading dimension ldg) and the Householder scalars
    auto launch_t = [&](const cx<T>* G, int ldg) -> int {
      const int nct = (int)ceil_div(kbo, TB_NT / 32);
      if (nb == TBB) {
        if (!g_tb_attr<T>) {
          QR_CUDA_TRY(cudaFuncSetAttribute(k_t_block<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)t_block_smem<T>(NBO)));
          g_tb_attr<T> = true;
        }
        QR_CUDA_TRY(launch_pdl(k_t_block<T>, dim3((unsigned)nct), dim3(TB_NT), t_block_smem<T>(kbo), st, Tb, nbo,
                               G, ldg, kbo));
      } else {
        if (!g_tc_attr<T>) {
          QR_CUDA_TRY(cudaFuncSetAttribute(k_t_cols<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)t_cols_smem<T>(NBO, NBO)));
          g_tc_attr<T> = true;
        }
        QR_CUDA_TRY(launch_pdl(k_t_cols<T>, dim3((unsigned)nct), dim3(TB_NT), t_cols_smem<T>(kbo, nct - 1), st,
                               Tb, nbo, G, ldg, static_cast<const cx<T>*>(s.tau + ko), kbo));
      }
      note_launch();
      return QRTEBD_OK;
    };
    // outer trailing update: C <- (I - V T V^dag)^dag C. With look-ahead the next outer
    // block's columns are updated here and the rest on the side stream, overlapping the
    // next block's panels.
    auto update = [&](int c0, int cw, cudaStream_t stream, cx<T>* W2, const QrGemm<T>* g) -> int {
      cx<T>* C = A + (long long)ko * lda + ko + kbo + c0;
      // W2 = T^dag V^dag C = (V T)^dag C, then C -= V W2
      GemmArgs<T> g1{kbo, cw, mo, VTb, 1, ldv, true, C, lda, 1, false, W2, cw, 1, one, zero};
      QR_TRY(run_gemm<T>(g1, s, stream, g));
      GemmArgs<T> g3{mo, cw, kbo, Vb, ldv, 1, false, W2, cw, 1, false, C, lda, 1, mone, one};
      QR_TRY(run_gemm<T>(g3, s, stream, g));
      return QRTEBD_OK;
    };
    // VT = V T of this block, for the trailing updates that take it
    auto form_vt = [&](cudaStream_t stream, const QrGemm<T>* g) -> int {
      GemmArgs<T> gv{mo, kbo, kbo, Vb, ldv, 1, false, Tb, nbo, 1, false, VTb, ldv, 1, one, zero};
      return run_gemm<T>(gv, s, stream, g);
    };
    // complex64 with look-ahead and a full next block: its 128 columns C1 are copied beside V
    // (into the next block's V storage, zero until its panels), one GEMM forms
    // [G | P] = V^dag [V | C1], T comes from G, and C1 -= V (T^dag P); V T, needed only by
    // the side stream's update (the explicit Q takes T_all), is formed there
    const bool gpf = qfast && kbo > nb && nc >= nbo;
    if (gpf) {
      cx<T>* C1 = A + (long long)ko * lda + ko + kbo;
      cx<T>* C1c = s.V + (long long)ko * ldv + ko + kbo;
      // C1 also carries block k-1's side-stream update: order after it
      if (latest(kblk - 1) >= 0) QR_CUDA_TRY(cudaStreamWaitEvent(st, ss->ev[nblk + latest(kblk - 1)], 0));
      QR_CUDA_TRY(cudaMemcpy2DAsync(C1c, (size_t)ldv * sizeof(cx<T>), C1, (size_t)lda * sizeof(cx<T>),
                                    (size_t)nbo * sizeof(cx<T>), (size_t)mo, cudaMemcpyDeviceToDevice, st));
      GemmArgs<T> ggp{kbo, kbo + nbo, mo, Vb, 1, ldv, true, Vb, ldv, 1, false, s.Wq, kbo + nbo, 1, one, zero};
      QR_TRY(run_gemm<T>(ggp, s, st, gm));
      // the next block's V is zero above its panels' diagonal blocks again
      QR_CUDA_TRY(cudaMemset2DAsync(C1c, (size_t)ldv * sizeof(cx<T>), 0, (size_t)nbo * sizeof(cx<T>),
                                    (size_t)std::min(mo, kbo + nbo), st));
      QR_TRY(launch_t(s.Wq, kbo + nbo));
      // a 128^3 product: the CUDA-core GEMM, which needs no operand preparation
      GemmArgs<T> gw{kbo, nbo, kbo, Tb, 1, nbo, true, s.Wq + kbo, kbo + nbo, 1, false, s.W2, nbo, 1, one, zero};
      QR_TRY(gemm_simt<T>(gw, st, s.gemm_scratch, s.gemm_scratch_elems));
      if (nc > nbo) {
        QR_CUDA_TRY(cudaEventRecord(ss->ev[kblk], st));  // V, T of this block are ready
        QR_CUDA_TRY(cudaStreamWaitEvent(ss->st, ss->ev[kblk], 0));
        QR_TRY(form_vt(ss->st, side));
        QR_TRY(update(nbo, nc - nbo, ss->st, s.W2s, side));
        QR_CUDA_TRY(cudaEventRecord(ss->ev[nblk + kblk], ss->st));
        rec[kblk] = 1;
      }
      GemmArgs<T> g3{mo, nbo, kbo, Vb, ldv, 1, false, s.W2, nbo, 1, false, C1, lda, 1, mone, one};
      QR_TRY(run_gemm<T>(g3, s, st, gm));
    } else {
      if (kbo > nb) {
        GemmArgs<T> gg{kbo, kbo, mo, Vb, 1, ldv, true, Vb, ldv, 1, false, s.G, nbo, 1, one, zero};
        QR_TRY(run_gemm<T>(gg, s, st, gm));
        QR_TRY(launch_t(s.G, nbo));
      }
      // V T for this block's updates, and for the backward explicit Q when T_all is not formed
      if (!qfast || nc > 0) QR_TRY(form_vt(st, gm));
      if (nc > 0) {
        // the next block's columns also carry block k-1's side-stream update: order after it
        if (ss && latest(kblk - 1) >= 0)
          QR_CUDA_TRY(cudaStreamWaitEvent(st, ss->ev[nblk + latest(kblk - 1)], 0));
        QR_TRY(update(0, n1, st, s.W2, gm));
        if (ss && nc > n1) {
          QR_CUDA_TRY(cudaEventRecord(ss->ev[kblk], st));  // V, T of this block are ready
          QR_CUDA_TRY(cudaStreamWaitEvent(ss->st, ss->ev[kblk], 0));
          QR_TRY(update(n1, nc - n1, ss->st, s.W2s, side));
          QR_CUDA_TRY(cudaEventRecord(ss->ev[nblk + kblk], ss->st));
          rec[kblk] = 1;
        }
      }
    }
    if (qfast) {
      // T_all's block column of this block, on the side stream:
      //   T_all[b, b] = T_b,  T_all[0:k, b] = -T_all[0:k, 0:k] (V[:, 0:k]^dag V_b) T_b
      // (V_b is zero above row ko, so the product runs over rows ko .. m-1)
      QR_CUDA_TRY(cudaEventRecord(ss->ev[2 * nblk + 2 + kblk], st));
      QR_CUDA_TRY(cudaStreamWaitEvent(ss->st, ss->ev[2 * nblk + 2 + kblk], 0));
      QR_CUDA_TRY(cudaMemcpy2DAsync(s.Tall + (long long)ko * n + ko, (size_t)n * sizeof(cx<T>), Tb,
                                    (size_t)nbo * sizeof(cx<T>), (size_t)kbo * sizeof(cx<T>), (size_t)kbo,
                                    cudaMemcpyDeviceToDevice, ss->st));
      if (ko > 0) {
        GemmArgs<T> gc{ko, kbo, mo, s.V + (long long)ko * ldv, 1, ldv, true, Vb, ldv, 1, false, s.Cb, kbo, 1,
                       one, zero};
        QR_TRY(run_gemm<T>(gc, s, ss->st, side));
        GemmArgs<T> gx{ko, kbo, kbo, s.Cb, kbo, 1, false, Tb, nbo, 1, false, s.Xb, kbo, 1, one, zero};
        QR_TRY(run_gemm<T>(gx, s, ss->st, side));
        GemmArgs<T> gt{ko, kbo, ko, s.Tall, n, 1, false, s.Xb, kbo, 1, false, s.Tall + ko, n, 1, mone, zero};
        QR_TRY(run_gemm<T>(gt, s, ss->st, side));
      }
    }
  }
  if (ss) {  // everything on the side stream (its updates, T_all) before the explicit Q
    QR_CUDA_TRY(cudaEventRecord(ss->ev[3 * nblk + 2], ss->st));
    QR_CUDA_TRY(cudaStreamWaitEvent(st, ss->ev[3 * nblk + 2], 0));
  }

  // explicit Q: with T_all, Q = -V W then its identity added; else backward accumulation
  // over the outer blocks from Q = [I; 0]
  if (!qfast) {
    long long tot = (long long)m * n;
    QR_CUDA_TRY(launch_pdl(k_eye<T>, dim3((unsigned)ceil_div(tot, 256)), dim3(256), 0, st, Q, ldq, m, n));
    note_launch();
    QR_CUDA_TRY(cudaGetLastError());
  }
  const int npo = qfast ? 0 : (int)ceil_div(n, nbo);
  if (qfast) {
    // Wq = T_all V_top^dag (V_top: the first n rows of V), then Q = [I; 0] - V Wq
    // V_top is unit lower triangular and T_all upper triangular (zeros stored in both), so
    // V_top^dag and Wq are upper triangular: both products stop each tile column's K loop
    // at its last column (the K-tiles skipped hold only zeros of the triangular factor)
    GemmArgs<T> gw{n, n, n, s.Tall, n, 1, false, s.V, 1, ldv, true, s.Wq, n, 1, one, zero};
    gw.tri_b = true;
    QR_TRY(run_gemm<T>(gw, s, st, gm));
    GemmArgs<T> gq{m, n, n, s.V, ldv, 1, false, s.Wq, n, 1, false, Q, ldq, 1, mone, zero};
    gq.tri_b = true;
    QR_TRY(run_gemm<T>(gq, s, st, gm));
    QR_CUDA_TRY(launch_pdl(k_add_eye<T>, dim3((unsigned)ceil_div(n, 256)), dim3(256), 0, st, Q, ldq, n));
    note_launch();
  }
  for (int p = npo - 1; p >= 0; --p) {
    const int ko = p * nbo;
    const int kbo = std::min(nbo, n - ko);
    const int mo = m - ko, nq = n - ko;
    const cx<T>* Vb = s.V + (long long)ko * ldv + ko;
    const cx<T>* VTb = s.VT + (long long)ko * ldv + ko;
    cx<T>* Qs = Q + (long long)ko * ldq + ko;
    // Q_s <- (I - V T V^dag) Q_s = Q_s - (V T)(V^dag Q_s)
    if (p == npo - 1) {
      // Q_s = [I; 0] here, so V^dag Q_s is the conjugate transpose of V's first nq rows:
      // one GEMM, Q_s -= (V T) V_top^dag
      GemmArgs<T> g0{mo, nq, kbo, VTb, ldv, 1, false, Vb, 1, ldv, true, Qs, ldq, 1, mone, one};
      QR_TRY(run_gemm<T>(g0, s, st, gm));
      continue;
    }
    GemmArgs<T> g1{kbo, nq, mo, Vb, 1, ldv, true, Qs, ldq, 1, false, s.W, nq, 1, one, zero};
    QR_TRY(run_gemm<T>(g1, s, st, gm));
    GemmArgs<T> g3{mo, nq, kbo, VTb, ldv, 1, false, s.W, nq, 1, false, Qs, ldq, 1, mone, one};
    QR_TRY(run_gemm<T>(g3, s, st, gm));
  }
  if (st != st_in) {  // join the caller's stream
    QR_CUDA_TRY(cudaEventRecord(ss->ev[2 * nblk + 1], st));
    QR_CUDA_TRY(cudaStreamWaitEvent(st_in, ss->ev[2 * nblk + 1], 0));
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
