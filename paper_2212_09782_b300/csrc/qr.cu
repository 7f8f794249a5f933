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

template <typename T> __host__ __device__ inline size_t panel_fixed_bytes() {
  return a16(2 * RED * sizeof(double)) + a16(2 * 16 * KBMAX * sizeof(cx<T>)) +
         2 * a16(KBMAX * sizeof(cx<T>)) + a16(4 * sizeof(cx<T>)) + a16(KBMAX * sizeof(cx<T>)) +
         a16(KBMAX * (KBMAX + 1) * sizeof(cx<T>));
}
template <typename T> __host__ __device__ inline size_t panel_smem_bytes(int rpc, int kb) {
  return a16((size_t)rpc * (kb + 1) * sizeof(cx<T>)) + a16((size_t)rpc * sizeof(cx<T>)) +
         panel_fixed_bytes<T>();
}

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

// Panel kernel. Per column j, two cluster-wide reductions, both push-style (each
// CTA stores its partial into slot [rank] of every CTA's buffer before the
// cluster barrier; after it all reads are local):
//   1. ||x||^2 below the pivot (FP64) and alpha;
//   2. w_c = v_j^dag P[:, c] for the columns c > j, and g_a = v_a^dag v_j for the
//      earlier reflectors a < j, which give column j of the compact-WY factor:
//      T(0:j, j) = -tau_j T(0:j, 0:j) g,  T(j, j) = tau_j.
// FP64 is used only for the norm and its square root (B300's FP64 pipe is narrow);
// the reflector scalars use Smith's complex division in the working precision.
template <typename T>
__global__ void __launch_bounds__(PT) k_qr_panel(PanelArgs<T> a) {
  extern __shared__ __align__(16) unsigned char sm[];
  cg::cluster_group cl = cg::this_cluster();
  const int CS = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = PT / 32;
  const int kb = a.kb, ldp = kb + 1, rpc = a.rpc;
  const int mr = a.m - a.k0;
  const int row0 = rank * rpc;
  const int nloc = max(0, min(rpc, mr - row0));

  unsigned char* q = sm;
  cx<T>* P = reinterpret_cast<cx<T>*>(q); q += a16((size_t)rpc * ldp * sizeof(cx<T>));
  cx<T>* VV = reinterpret_cast<cx<T>*>(q); q += a16((size_t)rpc * sizeof(cx<T>));
  double* red = reinterpret_cast<double*>(q); q += a16(2 * RED * sizeof(double));
  cx<T>* redT = reinterpret_cast<cx<T>*>(q); q += a16(2 * 16 * KBMAX * sizeof(cx<T>));
  cx<T>* wT = reinterpret_cast<cx<T>*>(q); q += a16(KBMAX * sizeof(cx<T>));
  cx<T>* gT = reinterpret_cast<cx<T>*>(q); q += a16(KBMAX * sizeof(cx<T>));
  cx<T>* bc = reinterpret_cast<cx<T>*>(q); q += a16(4 * sizeof(cx<T>));
  cx<T>* taus = reinterpret_cast<cx<T>*>(q); q += a16(KBMAX * sizeof(cx<T>));
  cx<T>* Ts = reinterpret_cast<cx<T>*>(q);  // KBMAX x (KBMAX + 1)

  const long long k0 = a.k0;
  for (int idx = tid; idx < nloc * kb; idx += PT) {
    const int p = idx / kb, c = idx % kb;
    P[p * ldp + c] = a.A[(k0 + row0 + p) * a.lda + k0 + c];
  }
  __syncthreads();

  for (int j = 0; j < kb; ++j) {
    const int buf = j & 1;
    // ---- reduction 1 (warp 0): ||x||^2 below the pivot in FP64, and alpha
    if (warp == 0) {
      double s = 0.0;
      T ar = 0, ai = 0;
      for (int p = lane; p < nloc; p += 32) {
        const int g = row0 + p;
        const cx<T> v = P[p * ldp + j];
        if (g > j) s = fma((double)v.x, (double)v.x, fma((double)v.y, (double)v.y, s));
        else if (g == j) { ar = v.x; ai = v.y; }
      }
      s = warp_sum(s);
      ar = warp_sum_t<T>(ar); ai = warp_sum_t<T>(ai);
      if (lane < CS) {
        double* dst = cl.map_shared_rank(red, lane) + buf * RED + 3 * rank;
        dst[0] = s; dst[1] = (double)ar; dst[2] = (double)ai;
      }
    }
    cl.sync();
    if (tid == 0) {
      double xn2 = 0;
      T alr = 0, ali = 0;
      const double* rr = red + buf * RED;
#pragma unroll 4
      for (int r = 0; r < CS; ++r) { xn2 += rr[3 * r]; alr += (T)rr[3 * r + 1]; ali += (T)rr[3 * r + 2]; }
      // zlarfg: beta = -sign(Re alpha) ||(alpha, x)||, tau = (beta - alpha) / beta,
      // v = x / (alpha - beta)
      T beta = alr, tr = 0, ti = 0, sr = 0, si = 0;
      if (!(xn2 == 0.0 && ali == T(0))) {
        const double nrm = sqrt(fma((double)alr, (double)alr, fma((double)ali, (double)ali, xn2)));
        beta = (T)(alr >= T(0) ? -nrm : nrm);
        tr = (beta - alr) / beta;
        ti = -ali / beta;
        // scale = 1 / (alpha - beta) by Smith's division (no squares of small numbers)
        const T dr = alr - beta, di = ali;
        if (fabs((double)dr) >= fabs((double)di)) {
          const T rt = di / dr, den = dr + di * rt;
          sr = T(1) / den; si = -rt / den;
        } else {
          const T rt = dr / di, den = di + dr * rt;
          sr = rt / den; si = T(-1) / den;
        }
      }
      if (!(isfinite((double)beta) && isfinite((double)sr) && isfinite((double)si)) && rank == 0)
        atomicOr(a.err, DEVERR_NUMERIC);
      bc[0] = mk<T>(beta, 0); bc[1] = mk<T>(tr, ti); bc[2] = mk<T>(sr, si);
      taus[j] = mk<T>(tr, ti);
    }
    __syncthreads();
    const T beta = bc[0].x;
    const cx<T> tau = bc[1], scale = bc[2];

    // ---- reduction 2: slots s < nc give w_{j+1+s}; slots s >= nc give g_{s-nc}
    const int nc = kb - j - 1;
    const int nslot = nc + j;
    if (nslot > 0) {
      for (int sl = warp; sl < nslot; sl += nwarps) {
        T wr = 0, wi = 0;
        const bool is_w = sl < nc;
        const int col = is_w ? j + 1 + sl : sl - nc;
        for (int p = lane; p < nloc; p += 32) {
          const int g = row0 + p;
          if (g < j) continue;
          const cx<T> v = (g == j) ? mk<T>(1, 0) : cmul<T>(P[p * ldp + j], scale);
          if (sl == 0) VV[p] = v;  // scaled reflector for the update pass
          const cx<T> x = P[p * ldp + col];
          if (is_w) { wr += v.x * x.x + v.y * x.y; wi += v.x * x.y - v.y * x.x; }   // conj(v) x
          else { wr += x.x * v.x + x.y * v.y; wi += x.x * v.y - x.y * v.x; }        // conj(v_a) v
        }
        wr = warp_sum_t<T>(wr); wi = warp_sum_t<T>(wi);
        if (lane < CS) cl.map_shared_rank(redT, lane)[buf * (KBMAX * 16) + rank * KBMAX + sl] = mk<T>(wr, wi);
      }
      cl.sync();
      if (tid < nslot) {
        cx<T> w = mk<T>(0, 0);
        const cx<T>* rr = redT + buf * (KBMAX * 16) + tid;
#pragma unroll 4
        for (int r = 0; r < CS; ++r) w = cadd<T>(w, rr[r * KBMAX]);
        if (tid < nc) wT[tid] = cmul<T>(cconj<T>(tau), w);  // conj(tau) w
        else gT[tid - nc] = w;
      }
      __syncthreads();
      if (warp == 0) {
        // T(0:j, j) = -tau_j T(0:j, 0:j) g ; T(j, j) = tau_j
        if (lane < j) {
          cx<T> acc = mk<T>(0, 0);
          for (int l = lane; l < j; ++l) cfma<T>(acc, Ts[lane * (KBMAX + 1) + l], gT[l]);
          const cx<T> r = cmul<T>(tau, acc);
          Ts[lane * (KBMAX + 1) + j] = mk<T>(-r.x, -r.y);
        }
        if (lane == 0) Ts[j * (KBMAX + 1) + j] = tau;
      }
      // P <- (I - conj(tau) v v^dag) P on columns c > j; column j <- v, pivot <- beta
      const int ncc = nc + 1;
      for (int idx = tid; idx < nloc * ncc; idx += PT) {
        const int p = idx / ncc, cc = idx % ncc;
        const int g = row0 + p;
        if (g < j) continue;
        if (cc == nc) {
          P[p * ldp + j] = (g > j) ? VV[p] : mk<T>(beta, T(0));
        } else {
          const cx<T> v = (g == j) ? mk<T>(1, 0) : VV[p];
          P[p * ldp + j + 1 + cc] = csub<T>(P[p * ldp + j + 1 + cc], cmul<T>(v, wT[cc]));
        }
      }
      __syncthreads();
    } else {
      // kb == 1: single column, no update and T = tau
      for (int p = tid; p < nloc; p += PT) {
        const int g = row0 + p;
        if (g > j) P[p * ldp + j] = cmul<T>(P[p * ldp + j], scale);
        else if (g == j) P[p * ldp + j] = mk<T>(beta, T(0));
      }
      if (tid == 0) Ts[0] = tau;
      __syncthreads();
    }
  }

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
  cl.sync();  // no CTA leaves while others may still store into its shared memory
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
                   QrScratch<T>& s, cudaStream_t st, unsigned* err, const QrGemm<T>* gm) {
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

  for (int ko = 0; ko < n; ko += nbo) {
    const int kbo = std::min(nbo, n - ko);
    const int mo = m - ko;
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
    // outer trailing update: C <- (I - V T V^dag)^dag C
    const int nc = n - ko - kbo;
    if (nc > 0) {
      cx<T>* C = A + (long long)ko * lda + ko + kbo;
      GemmArgs<T> g1{kbo, nc, mo, Vb, 1, ldv, true, C, lda, 1, false, s.W, nc, 1, one, zero};
      QR_TRY(run_gemm<T>(g1, s, st, gm));
      GemmArgs<T> g2{kbo, nc, kbo, Tb, 1, nbo, true, s.W, nc, 1, false, s.W2, nc, 1, one, zero};
      QR_TRY(run_gemm<T>(g2, s, st, gm));
      GemmArgs<T> g3{mo, nc, kbo, Vb, ldv, 1, false, s.W2, nc, 1, false, C, lda, 1, mone, one};
      QR_TRY(run_gemm<T>(g3, s, st, gm));
    }
  }

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
                                   QrScratch<float>&, cudaStream_t, unsigned*, const QrGemm<float>*);
template int householder_qr<double>(double2*, long long, int, int, double2*, long long,
                                    QrScratch<double>&, cudaStream_t, unsigned*, const QrGemm<double>*);

}  // namespace qrtebd
