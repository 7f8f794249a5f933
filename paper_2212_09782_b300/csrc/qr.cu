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
constexpr int RED = 2 * KBMAX + 4;
constexpr int SMEM_CAP = 220 * 1024;

template <typename T> struct PanelArgs {
  cx<T>* A; long long lda; int m; int k0; int kb;
  cx<T>* V; long long ldv;
  cx<T>* tau; cx<T>* Tf; int ldt;
  int rpc; unsigned* err;
};

__host__ __device__ inline size_t a16(size_t x) { return (x + 15) & ~size_t(15); }

template <typename T> __host__ __device__ inline size_t panel_fixed_bytes() {
  return a16(2 * RED * sizeof(double)) + a16(RED * sizeof(double)) +
         2 * a16(KBMAX * KBMAX * sizeof(double)) + a16(32 * sizeof(double)) +
         a16(KBMAX * sizeof(cx<T>)) + a16(KBMAX * (KBMAX + 1) * sizeof(cx<T>));
}
template <typename T> __host__ __device__ inline size_t panel_smem_bytes(int rpc, int kb) {
  return a16((size_t)rpc * (kb + 1) * sizeof(cx<T>)) + panel_fixed_bytes<T>();
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

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
  double* red = reinterpret_cast<double*>(q); q += a16(2 * RED * sizeof(double));
  double* bc = reinterpret_cast<double*>(q); q += a16(RED * sizeof(double));
  double* gp_ = reinterpret_cast<double*>(q); q += a16(KBMAX * KBMAX * sizeof(double));
  double* gsum = reinterpret_cast<double*>(q); q += a16(KBMAX * KBMAX * sizeof(double));
  double* wsum = reinterpret_cast<double*>(q); q += a16(32 * sizeof(double));
  cx<T>* taus = reinterpret_cast<cx<T>*>(q); q += a16(KBMAX * sizeof(cx<T>));
  cx<T>* Ts = reinterpret_cast<cx<T>*>(q);

  const long long k0 = a.k0;
  for (int idx = tid; idx < nloc * kb; idx += PT) {
    int p = idx / kb, c = idx % kb;
    P[p * ldp + c] = a.A[(k0 + row0 + p) * a.lda + k0 + c];
  }
  __syncthreads();

  int buf = 0;
  for (int j = 0; j < kb; ++j) {
    // ---- reduction 1: ||x||^2 (rows below the pivot) in FP64, plus alpha
    double s = 0.0, ar = 0.0, ai = 0.0;
    for (int p = tid; p < nloc; p += PT) {
      int g = row0 + p;
      cx<T> v = P[p * ldp + j];
      if (g > j) s += (double)v.x * v.x + (double)v.y * v.y;
      else if (g == j) { ar = v.x; ai = v.y; }
    }
    s = warp_sum(s); ar = warp_sum(ar); ai = warp_sum(ai);
    if (lane == 0) { wsum[warp * 4 + 0] = s; wsum[warp * 4 + 1] = ar; wsum[warp * 4 + 2] = ai; }
    __syncthreads();
    if (tid == 0) {
      double t0 = 0, t1 = 0, t2 = 0;
      for (int w = 0; w < nwarps; ++w) { t0 += wsum[w * 4]; t1 += wsum[w * 4 + 1]; t2 += wsum[w * 4 + 2]; }
      red[buf * RED + 0] = t0; red[buf * RED + 1] = t1; red[buf * RED + 2] = t2;
    }
    cl.sync();
    if (warp == 0) {
      double t0 = 0, t1 = 0, t2 = 0;
      if (lane < CS) {
        const double* r = cl.map_shared_rank(red, lane) + buf * RED;
        t0 = r[0]; t1 = r[1]; t2 = r[2];
      }
      t0 = warp_sum(t0); t1 = warp_sum(t1); t2 = warp_sum(t2);
      if (lane == 0) { bc[0] = t0; bc[1] = t1; bc[2] = t2; }
    }
    __syncthreads();
    buf ^= 1;
    const double xn2 = bc[0], alr = bc[1], ali = bc[2];
    double beta, tr, ti, sr, si;
    if (xn2 == 0.0 && ali == 0.0) {
      beta = alr; tr = 0.0; ti = 0.0; sr = 0.0; si = 0.0;
    } else {
      beta = -copysign(sqrt(alr * alr + ali * ali + xn2), alr);
      tr = (beta - alr) / beta; ti = -ali / beta;
      double dr = alr - beta, di = ali, den = dr * dr + di * di;
      sr = dr / den; si = -di / den;
    }
    if (!isfinite(beta) && tid == 0 && rank == 0) atomicOr(a.err, DEVERR_NUMERIC);
    const cx<T> scale = mk<T>((T)sr, (T)si);
    for (int p = tid; p < nloc; p += PT) {
      int g = row0 + p;
      if (g > j) P[p * ldp + j] = cmul<T>(P[p * ldp + j], scale);
      else if (g == j) P[p * ldp + j] = mk<T>((T)beta, (T)0);
    }
    if (tid == 0) taus[j] = mk<T>((T)tr, (T)ti);
    __syncthreads();

    // ---- reduction 2: w_c = sum_{g >= j} conj(v_g) P[g][c], c > j
    const int nc = kb - j - 1;
    if (nc > 0) {
      for (int c = j + 1 + warp; c < kb; c += nwarps) {
        T wr = 0, wi = 0;
        for (int p = lane; p < nloc; p += 32) {
          int g = row0 + p;
          if (g < j) continue;
          cx<T> v = (g == j) ? mk<T>(1, 0) : P[p * ldp + j];
          cx<T> x = P[p * ldp + c];
          wr += v.x * x.x + v.y * x.y;
          wi += v.x * x.y - v.y * x.x;
        }
        double dwr = warp_sum((double)wr), dwi = warp_sum((double)wi);
        if (lane == 0) { red[buf * RED + 2 * (c - j - 1)] = dwr; red[buf * RED + 2 * (c - j - 1) + 1] = dwi; }
      }
      cl.sync();
      if (tid < nc) {
        double wr = 0, wi = 0;
        for (int r = 0; r < CS; ++r) {
          const double* rr = cl.map_shared_rank(red, r) + buf * RED;
          wr += rr[2 * tid]; wi += rr[2 * tid + 1];
        }
        bc[4 + 2 * tid] = wr; bc[4 + 2 * tid + 1] = wi;
      }
      __syncthreads();
      buf ^= 1;
      // P <- (I - conj(tau) v v^dag) P on columns c > j
      const cx<T> ctau = mk<T>((T)tr, (T)-ti);
      for (int idx = tid; idx < nloc * nc; idx += PT) {
        int p = idx / nc, cc = idx % nc;
        int g = row0 + p;
        if (g < j) continue;
        cx<T> v = (g == j) ? mk<T>(1, 0) : P[p * ldp + j];
        cx<T> w = mk<T>((T)bc[4 + 2 * cc], (T)bc[4 + 2 * cc + 1]);
        cx<T> t = cmul<T>(ctau, w);
        P[p * ldp + j + 1 + cc] = csub<T>(P[p * ldp + j + 1 + cc], cmul<T>(v, t));
      }
      __syncthreads();
    }
  }

  // ---- compact-WY T from G = V^dag V (strictly upper part)
  const int npairs = kb * (kb - 1) / 2;
  for (int idx = tid; idx < npairs; idx += PT) {
    int b = (int)((1.0 + sqrt(1.0 + 8.0 * idx)) * 0.5);
    while (b * (b - 1) / 2 > idx) --b;
    while ((b + 1) * b / 2 <= idx) ++b;
    int aa = idx - b * (b - 1) / 2;
    T gr = 0, gi = 0;
    for (int p = max(0, b - row0); p < nloc; ++p) {
      // v_b is zero above row b (and v_a above row a < b)
      int g = row0 + p;
      cx<T> va = P[p * ldp + aa];
      cx<T> vb = (g == b) ? mk<T>(1, 0) : P[p * ldp + b];
      gr += va.x * vb.x + va.y * vb.y;
      gi += va.x * vb.y - va.y * vb.x;
    }
    gp_[2 * idx] = (double)gr; gp_[2 * idx + 1] = (double)gi;
  }
  cl.sync();
  if (rank == 0) {
    for (int idx = tid; idx < npairs; idx += PT) {
      double gr = 0, gi = 0;
      for (int r = 0; r < CS; ++r) {
        const double* rr = cl.map_shared_rank(gp_, r);
        gr += rr[2 * idx]; gi += rr[2 * idx + 1];
      }
      gsum[2 * idx] = gr; gsum[2 * idx + 1] = gi;
    }
    __syncthreads();
    if (warp == 0) {
      // T(0:j, j) = -tau_j T(0:j, 0:j) G(0:j, j); T(j, j) = tau_j
      for (int j = 0; j < kb; ++j) {
        cx<T> tj = taus[j];
        if (lane < j) {
          double sr2 = 0, si2 = 0;
          for (int l = lane; l < j; ++l) {
            cx<T> t = Ts[lane * (KBMAX + 1) + l];
            int pi = j * (j - 1) / 2 + l;
            double gr = gsum[2 * pi], gi = gsum[2 * pi + 1];
            sr2 += (double)t.x * gr - (double)t.y * gi;
            si2 += (double)t.x * gi + (double)t.y * gr;
          }
          double rr = -((double)tj.x * sr2 - (double)tj.y * si2);
          double ri = -((double)tj.x * si2 + (double)tj.y * sr2);
          Ts[lane * (KBMAX + 1) + j] = mk<T>((T)rr, (T)ri);
        } else if (lane == j) {
          Ts[j * (KBMAX + 1) + j] = tj;
        }
        __syncwarp();
      }
    }
    __syncthreads();
    for (int idx = tid; idx < kb * kb; idx += PT) {
      int i = idx / kb, j = idx % kb;
      a.Tf[i * a.ldt + j] = (j >= i) ? Ts[i * (KBMAX + 1) + j] : mk<T>(0, 0);
    }
    if (tid < kb) a.tau[k0 + tid] = taus[tid];
  }

  // ---- write V (explicit, unit lower trapezoidal) and R / zeros into A
  for (int idx = tid; idx < nloc * kb; idx += PT) {
    int p = idx / kb, c = idx % kb;
    int g = row0 + p;
    cx<T> pv = P[p * ldp + c];
    cx<T> v = (g == c) ? mk<T>(1, 0) : (g > c ? pv : mk<T>(0, 0));
    a.V[(k0 + g) * a.ldv + k0 + c] = v;
    a.A[(k0 + g) * a.lda + k0 + c] = (c >= g) ? pv : mk<T>(0, 0);
  }
  cl.sync();  // keep shared memory alive until every remote read has finished
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
  // sized for the widest panel: ceil(n/nb) * nb * nb <= (n + KBMAX) * KBMAX for any nb <= KBMAX
  const int nb = KBMAX;
  s.V = ar.take<cx<T>>((size_t)m * n);
  s.tau = ar.take<cx<T>>(n);
  s.Tf = ar.take<cx<T>>((size_t)(n + nb) * nb);
  s.W = ar.take<cx<T>>((size_t)nb * n);
  s.W2 = ar.take<cx<T>>((size_t)nb * n);
  size_t e1 = gemm_simt_scratch_elems(nb, n, m, 1);
  size_t e2 = gemm_simt_scratch_elems(m, n, nb, 1);
  s.gemm_scratch_elems = e1 > e2 ? e1 : e2;
  s.gemm_scratch = s.gemm_scratch_elems ? ar.take<cx<T>>(s.gemm_scratch_elems) : nullptr;
}

template <typename T>
int householder_qr(cx<T>* A, long long lda, int m, int n, cx<T>* Q, long long ldq,
                   QrScratch<T>& s, cudaStream_t st, unsigned* err, const QrGemm<T>* gm) {
  if (m < n || n < 1) return QRTEBD_ERR_INVALID_ARG;
  QR_TRY(probe_max_cluster<T>());
  const int nb = qr_panel_width(m, n, sizeof(cx<T>));
  if (nb < 1) { set_last_message("QR: matrix too tall for the shared-memory panel"); return QRTEBD_ERR_INVALID_ARG; }
  const long long ldv = n;
  const cx<T> one = mk<T>(1, 0), zero = mk<T>(0, 0), mone = mk<T>(-1, 0);

  for (int k0 = 0; k0 < n; k0 += nb) {
    const int kb = std::min(nb, n - k0);
    const int mr = m - k0;
    ClusterChoice cc = choose_cluster<T>(mr, kb);
    if (cc.cs < 0 || cc.kb != kb) {
      cc.kb = kb;  // kb was validated at k0 = 0 (largest mr); recompute rows per CTA
      cc.cs = 16; cc.rpc = (int)ceil_div(mr, 16);
    }
    PanelArgs<T> pa{A, lda, m, k0, kb, s.V, ldv, s.tau, s.Tf + (size_t)(k0 / nb) * nb * nb, nb,
                    cc.rpc, err};
    QR_TRY(launch_panel<T>(pa, cc.cs, st));
    const int nc = n - k0 - kb;
    if (nc > 0) {
      const cx<T>* Vk = s.V + (long long)k0 * ldv + k0;
      cx<T>* C = A + (long long)k0 * lda + k0 + kb;
      const cx<T>* Tk = s.Tf + (size_t)(k0 / nb) * nb * nb;
      // W = V^dag C  (kb x nc)
      GemmArgs<T> g1{kb, nc, mr, Vk, 1, ldv, true, C, lda, 1, false, s.W, nc, 1, one, zero};
      QR_TRY(run_gemm<T>(g1, s, st, gm));
      // W2 = T^dag W
      GemmArgs<T> g2{kb, nc, kb, Tk, 1, nb, true, s.W, nc, 1, false, s.W2, nc, 1, one, zero};
      QR_TRY(run_gemm<T>(g2, s, st, gm));
      // C -= V W2
      GemmArgs<T> g3{mr, nc, kb, Vk, ldv, 1, false, s.W2, nc, 1, false, C, lda, 1, mone, one};
      QR_TRY(run_gemm<T>(g3, s, st, gm));
    }
  }

  // explicit Q by backward accumulation
  {
    long long tot = (long long)m * n;
    k_eye<T><<<(unsigned)ceil_div(tot, 256), 256, 0, st>>>(Q, ldq, m, n);
    note_launch();
    QR_CUDA_TRY(cudaGetLastError());
  }
  const int np = (int)ceil_div(n, nb);
  for (int p = np - 1; p >= 0; --p) {
    const int k0 = p * nb;
    const int kb = std::min(nb, n - k0);
    const int mr = m - k0, nq = n - k0;
    const cx<T>* Vk = s.V + (long long)k0 * ldv + k0;
    const cx<T>* Tk = s.Tf + (size_t)p * nb * nb;
    cx<T>* Qs = Q + (long long)k0 * ldq + k0;
    GemmArgs<T> g1{kb, nq, mr, Vk, 1, ldv, true, Qs, ldq, 1, false, s.W, nq, 1, one, zero};
    QR_TRY(run_gemm<T>(g1, s, st, gm));
    GemmArgs<T> g2{kb, nq, kb, Tk, nb, 1, false, s.W, nq, 1, false, s.W2, nq, 1, one, zero};
    QR_TRY(run_gemm<T>(g2, s, st, gm));
    GemmArgs<T> g3{mr, nq, kb, Vk, ldv, 1, false, s.W2, nq, 1, false, Qs, ldq, 1, mone, one};
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
