// One QR-TEBD bond update on the device; see bond.cuh and qrtebd.h.
//
// Step order (Sec. II, Fig. 2b; Sec. III, Fig. 3):
//   (i)   theta' = B^m B^n (skipped when theta' is given), theta~' = U theta',
//         theta~ = Xi theta~', Y0 per the eta policy, X = theta~ Y0^dag, QR(X) -> Q
//   (ii)  Z = Y^dag = theta~^dag Q, QR(Z) -> Qz, Rz  (LQ of Y: L = Rz^dag, Q^[n] = Qz^dag)
//   (iv)  CBE only: L^dag L = Rz Rz^dag = V^dag S^2 V (Jacobi, FP64), cut to chi~
//   (iii/v) B~^n = Q^[n] (PLAIN) or P V Q^[n] (CBE); Xi~ = L or diag(S) normalised;
//         B~^m = theta~' B~^n^dag (Hastings form)
//   eps   = 1 - kept / ||theta~||^2 with both norms accumulated in FP64; for
//         orthogonal projectors this equals ||theta~ - approx||^2 / ||theta~||^2.
#include "bond.cuh"
#include "tc_gemm.cuh"

namespace qrtebd {

namespace {

constexpr int RED_BLOCKS = 592;  // 4 x 148 SMs

// ------------------------------------------------------------------ gate
// theta~'[a, i, j, b] = sum_{k,l} U[(i j), (k l)] theta'[a, k, l, b]; one thread
// per (a, b), the d^2 inputs in registers, U in shared memory. Optionally also
// writes theta~ = diag(xi) theta~' (Xi diagonal).
template <typename T, int D>
__global__ void k_gate(const cx<T>* __restrict__ th, cx<T>* __restrict__ out,
                       const double2* __restrict__ U, int chiL, int chiR,
                       const cx<T>* __restrict__ xi_diag, cx<T>* __restrict__ out_xi) {
  constexpr int D2 = D * D;
  __shared__ cx<T> Us[D2 * D2];
  for (int t = threadIdx.x; t < D2 * D2; t += blockDim.x) {
    double2 u = U[t];
    Us[t] = mk<T>((T)u.x, (T)u.y);
  }
  __syncthreads();
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)chiL * chiR) return;
  long long a = idx / chiR, b = idx % chiR;
  long long base = a * D2 * chiR + b;
  cx<T> in[D2];
#pragma unroll
  for (int q = 0; q < D2; ++q) in[q] = th[base + (long long)q * chiR];
  cx<T> xa = xi_diag ? xi_diag[a] : mk<T>(1, 0);
#pragma unroll
  for (int o = 0; o < D2; ++o) {
    cx<T> acc = mk<T>(0, 0);
#pragma unroll
    for (int q = 0; q < D2; ++q) cfma<T>(acc, Us[o * D2 + q], in[q]);
    out[base + (long long)o * chiR] = acc;
    if (out_xi) out_xi[base + (long long)o * chiR] = cmul<T>(xa, acc);
  }
}

template <typename T>
__global__ void k_convert_gate(const double2* U, cx<T>* Ut, int n) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) Ut[t] = mk<T>((T)U[t].x, (T)U[t].y);
}

template <typename T>
__global__ void k_scale_rows(const cx<T>* in, cx<T>* out, const cx<T>* xi, long long rows,
                             long long rowlen) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= rows * rowlen) return;
  out[idx] = cmul<T>(xi[idx / rowlen], in[idx]);
}

// ------------------------------------------------------------------ norms
template <typename T>
__global__ void k_norm2_partial(const cx<T>* __restrict__ x, long long n, double* partial) {
  double s = 0.0;
  if constexpr (std::is_same<T, float>::value) {
    // complex64: each thread accumulates in double-float (exact FP32 squares by FMA,
    // TwoSum additions, ~48-bit significand) and only its total goes to FP64: per-element
    // FP64 arithmetic made this pass FP64-bound on B300 (~4x its memory time)
    float hi = 0.f, lo = 0.f;
    auto add_sq = [&](float v) {
      const float p = v * v, e = fmaf(v, v, -p);
      const float t = hi + p, bb = t - hi;
      const float err = (hi - (t - bb)) + (p - bb);
      const float l = lo + err + e;
      hi = t + l;
      lo = l - (hi - t);
    };
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
      const cx<T> v = x[i];
      add_sq(v.x);
      add_sq(v.y);
    }
    s = (double)hi + (double)lo;
  } else {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
      cx<T> v = x[i];
      s += (double)v.x * v.x + (double)v.y * v.y;
    }
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ double ws[32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
    partial[blockIdx.x] = t;
  }
}

// Deterministic final sum (fixed order) into *out.
__global__ void k_sum_partials(const double* partial, int n, double* out) {
  __shared__ double ws[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += partial[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
    *out = t;
  }
}

// stats = {eps, ||theta~||^2, kept, chi_new}; scal[0] = 1/sqrt(kept_norm), the scale that
// normalises the kept values (kept_norm: nullptr = kept)
__global__ void k_finalize(const double* th2, const double* kept, double chi_new, double* stats,
                           double* scal, unsigned* err, const double* kept_norm = nullptr,
                           const int* chi_dev = nullptr) {
  double t = *th2, k = *kept, kn = kept_norm ? *kept_norm : k;
  double eps = t > 0 ? 1.0 - k / t : 0.0;
  if (eps < 0) eps = 0;
  if (!isfinite(t) || !isfinite(k) || !isfinite(kn)) atomicOr(err, DEVERR_NUMERIC);
  if (stats) { stats[0] = eps; stats[1] = t; stats[2] = k; stats[3] = chi_dev ? (double)*chi_dev : chi_new; }
  scal[0] = kn > 0 ? 1.0 / sqrt(kn) : 0.0;
}

// ---- the CBE tail with the cut chi~ on the device (chi = *chi_dev, n the expansion eta)
// Vt = V with its rows from chi~ on zeroed (the projector P of step (v)), n x n
template <typename T> __global__ void k_from_c128_rows(const double2* in, cx<T>* out, int n, const int* chi_dev) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= (long long)n * n) return;
  const int c = *chi_dev;
  out[i] = (i / n < c) ? mk<T>((T)in[i].x, (T)in[i].y) : mk<T>(0, 0);
}
// dst[0 : chi~ cols) = src[0 : chi~ cols): the first chi~ rows of a row-major matrix
template <typename T> __global__ void k_copy_rows_dev(const cx<T>* src, cx<T>* dst, long long cols, int n, const int* chi_dev) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= (long long)n * cols) return;
  if (i < (long long)*chi_dev * cols) dst[i] = src[i];
}
// dst (rows x chi~, leading dimension chi~) = the first chi~ columns of src (leading dimension n)
template <typename T> __global__ void k_copy_cols_dev(const cx<T>* src, int n, cx<T>* dst, long long rows, const int* chi_dev) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= rows * n) return;
  const int c = *chi_dev;
  const long long r = i / n;
  const int j = (int)(i % n);
  if (j < c) dst[r * c + j] = src[i];
}
// Xi~ = diag(S[0 : chi~]) / ||.|| as a dense chi~ x chi~ matrix (grid over n x n)
template <typename T> __global__ void k_diag_xi_dev(const double* S, const int* chi_dev, int n, const double* scal, cx<T>* xi) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int c = *chi_dev;
  if (idx >= (long long)c * c || idx >= (long long)n * n) return;
  const int i = (int)(idx / c), j = (int)(idx % c);
  xi[idx] = mk<T>(i == j ? (T)(S[i] * scal[0]) : T(0), 0);
}

// explicit eps = ||theta~ - approx||^2 / ||theta~||^2 overrides stats[0]
__global__ void k_eps_explicit(const double* th2, const double* r2, double* stats) {
  double t = *th2;
  stats[0] = t > 0 ? *r2 / t : 0.0;
}

// out[j][i] = s * conj(in[i][j]) for i < rows, j < cols (in: ld_in, out: ld_out)
template <typename T>
__global__ void k_conj_transpose(const cx<T>* in, long long ld_in, cx<T>* out, long long ld_out,
                                 int rows, int cols, const double* scale) {
  __shared__ cx<T> tile[32][33];
  int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
  T s = scale ? (T)scale[0] : T(1);
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    int i = i0 + r, j = j0 + threadIdx.x;
    if (i < rows && j < cols) tile[r][threadIdx.x] = in[i * ld_in + j];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    int j = j0 + r, i = i0 + threadIdx.x;
    if (i < rows && j < cols) {
      cx<T> v = tile[threadIdx.x][r];
      out[j * ld_out + i] = mk<T>(s * v.x, -s * v.y);
    }
  }
}

template <typename T>
int conj_transpose(const cx<T>* in, long long ld_in, cx<T>* out, long long ld_out, int rows,
                   int cols, const double* scale, cudaStream_t st) {
  dim3 grid((unsigned)ceil_div(cols, 32), (unsigned)ceil_div(rows, 32));
  k_conj_transpose<T><<<grid, dim3(32, 8), 0, st>>>(in, ld_in, out, ld_out, rows, cols, scale);
  note_launch();
  QR_CUDA_TRY(cudaGetLastError());
  return QRTEBD_OK;
}

template <typename T>
int norm2(const cx<T>* x, long long n, double* partial, double* out, cudaStream_t st) {
  k_norm2_partial<T><<<RED_BLOCKS, 256, 0, st>>>(x, n, partial);
  note_launch();
  QR_CUDA_TRY(cudaGetLastError());
  k_sum_partials<<<1, 256, 0, st>>>(partial, RED_BLOCKS, out);
  note_launch();
  QR_CUDA_TRY(cudaGetLastError());
  return QRTEBD_OK;
}

template <typename T>
int launch_gate(const cx<T>* th, cx<T>* out, const double2* U, int chiL, int d, int chiR,
                const cx<T>* xi_diag, cx<T>* out_xi, cudaStream_t st) {
  long long n = (long long)chiL * chiR;
  unsigned grid = (unsigned)ceil_div(n, 128);
  ProfScope prof(PROF_GATE, st, 8.0 * n * d * d * d * d,
                 (double)sizeof(cx<T>) * n * d * d * (out_xi ? 3 : 2));
  switch (d) {
#define QR_GATE_CASE(DD) \
    case DD: k_gate<T, DD><<<grid, 128, 0, st>>>(th, out, U, chiL, chiR, xi_diag, out_xi); note_launch(); break;
    QR_GATE_CASE(2) QR_GATE_CASE(3) QR_GATE_CASE(4) QR_GATE_CASE(5)
#undef QR_GATE_CASE
    default: return QRTEBD_ERR_INVALID_ARG;
  }
  QR_CUDA_TRY(cudaGetLastError());
  return QRTEBD_OK;
}

// ------------------------------------------------------------------ CBE cut
// Reads w (descending eigenvalues of L^dag L), writes S = sqrt(max(w, 0)),
// decides chi~ (Fig. 4 caption: drop S / ||S|| < svd_min, keep <= chi_max, never
// split a multiplet closer than tie_tol * S_1), kept = sum_{k < chi~} S_k^2.
// The cut of Sec. III (svd_min, chi_max, eps_target, then the tie rule). kept (for eps):
// ||L||^2 - sum of the discarded S^2, with ||L||^2 = lnorm2 summed in FP64 from L itself:
// the discarded values are accurate relative to themselves, whereas the sum of the kept
// ones carries the decomposition's rounding relative to the largest (~1e-6 for the FP32
// solver at eta ~ 1000) into eps, which is itself ~1e-6 per update at chi ~ 1000.
// kept_norm: the sum of the kept S^2, which normalises Xi~ exactly.
__global__ void k_cbe_cut(const double* w, int n, int chi_max, double svd_min, double tie_tol,
                          double eps_target, const double* lnorm2, double* S, double* kept,
                          double* kept_norm, int* chi_out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double tot = 0;
  for (int k = 0; k < n; ++k) { double s = w[k] > 0 ? sqrt(w[k]) : 0.0; S[k] = s; tot += s * s; }
  if (*lnorm2 > 0) tot = *lnorm2;
  double nrm = sqrt(tot);
  int c = 0;
  if (nrm > 0) { for (int k = 0; k < n; ++k) if (S[k] / nrm >= svd_min) ++c; }
  if (c > chi_max) c = chi_max;
  if (c < 1) c = 1;
  if (eps_target > 0 && tot > 0) {
    // fewest values whose discarded weight (relative to the total) is <= eps_target
    double tail = 0;
    int ce = n;
    while (ce > 1 && tail + S[ce - 1] * S[ce - 1] <= eps_target * tot) { tail += S[ce - 1] * S[ce - 1]; --ce; }
    if (ce < c) c = ce;
  }
  if (nrm > 0) {
    while (c < n && c > 1 && (S[c - 1] - S[c]) / nrm <= tie_tol * (S[0] / nrm)) --c;
  }
  double kk = 0, tail = 0;
  for (int k = 0; k < c; ++k) kk += S[k] * S[k];
  for (int k = n - 1; k >= c; --k) tail += S[k] * S[k];  // smallest first
  *kept = tot - tail;
  *kept_norm = kk;
  *chi_out = c;
}

// D = v * identity (n x n)
template <typename T> __global__ void k_scaled_eye(cx<T>* D, int n, T v) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)n * n) return;
  D[idx] = mk<T>(idx / n == idx % n ? v : T(0), T(0));
}

template <typename T> __global__ void k_to_c128(const cx<T>* in, double2* out, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) out[i] = make_double2((double)in[i].x, (double)in[i].y);
}
template <typename T> __global__ void k_from_c128(const double2* in, cx<T>* out, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) out[i] = mk<T>((T)in[i].x, (T)in[i].y);
}

// ------------------------------------------------------------------ driver
template <typename T>
struct GemmRunner {
  // Routes a GEMM either to CUDA cores or (complex64 tensor-core precisions) to tcgen05.
  int precision;
  TcWorkspace* tc;
  cx<T>* simt_scratch;
  size_t simt_scratch_elems;
  OzWorkspace* oz = nullptr;  // complex128 with FP64 emulated on the tensor cores
  // bond: a bond-level contraction (profiled as PROF_BOND_GEMM), else a QR-internal one
  int run(const GemmArgs<T>& g, cudaStream_t st, bool bond = false) const;
};

template <>
int GemmRunner<double>::run(const GemmArgs<double>& g, cudaStream_t st, bool bond) const {
  if (precision == QRTEBD_C128_OZ && oz && oz_gemm_eligible(g))
    return oz_gemm(g, *oz, st, bond ? PROF_BOND_GEMM : PROF_TC_GEMM);
  return gemm_simt<double>(g, st, simt_scratch, simt_scratch_elems,
                           bond ? PROF_BOND_GEMM : PROF_SIMT_GEMM);
}
template <>
int GemmRunner<float>::run(const GemmArgs<float>& g, cudaStream_t st, bool bond) const {
  if ((precision == QRTEBD_C64_3XTF32 || precision == QRTEBD_C64_TF32) && tc &&
      tc_gemm_eligible(g)) {
    return tc_gemm(g, precision == QRTEBD_C64_3XTF32, *tc, st, bond ? PROF_BOND_GEMM : PROF_TC_GEMM);
  }
  return gemm_simt<float>(g, st, simt_scratch, simt_scratch_elems,
                          bond ? PROF_BOND_GEMM : PROF_SIMT_GEMM);
}

template <typename T> int qr_gemm_thunk(const GemmArgs<T>& g, cudaStream_t st, void* ctx) {
  return static_cast<const GemmRunner<T>*>(ctx)->run(g, st);
}

template <typename T>
int bond_update_t(const qrtebd_bond_io* io, const qrtebd_trunc* tr, cudaStream_t st,
                  qrtebd_bond_info* info, size_t* bytes, bool sync_chi, bool theta_gated) {
  const int chiL = io->chi_l, d = io->d, chiM = io->chi_m, chiR = io->chi_r;
  const bool measuring = (bytes != nullptr);
  const long long mL = (long long)chiL * d, nR = (long long)d * chiR;
  const int eta = choose_eta(tr, chiL, d, chiM, chiR);
  if (eta < 1) { set_last_message("bond_update: eta out of range"); return QRTEBD_ERR_INVALID_ARG; }
  const bool cbe = (tr->scheme == QRTEBD_CBE);
  const bool theta_given = (io->theta != nullptr) || (measuring && io->bm == nullptr);
  const bool y0_is_bn = (!cbe && eta == chiM);
  const bool use_tc = std::is_same<T, float>::value &&
                      (io->precision == QRTEBD_C64_3XTF32 || io->precision == QRTEBD_C64_TF32);

  Arena ar;
  ar.measuring = measuring;
  if (!measuring) { ar.base = static_cast<char*>(io->workspace); ar.cap = io->workspace_bytes; }

  cx<T>* theta_p = theta_given ? nullptr : ar.take<cx<T>>((size_t)mL * nR);
  // theta_gated: io->theta already holds theta~' = U theta' (read only from here on)
  cx<T>* theta_tp = theta_gated ? const_cast<cx<T>*>(static_cast<const cx<T>*>(io->theta))
                                : ar.take<cx<T>>((size_t)mL * nR);
  cx<T>* theta_t = (io->xi_kind == 0) ? theta_tp : ar.take<cx<T>>((size_t)mL * nR);
  cx<T>* X = ar.take<cx<T>>((size_t)mL * eta);
  cx<T>* Q = ar.take<cx<T>>((size_t)mL * eta);
  cx<T>* Z = ar.take<cx<T>>((size_t)nR * eta);
  cx<T>* Qz = ar.take<cx<T>>((size_t)nR * eta);
  cx<T>* Ut = (d > 5 && !theta_gated) ? ar.take<cx<T>>((size_t)d * d * d * d) : nullptr;
  QrScratch<T> qs;
  qr_carve<T>(ar, (int)std::max(mL, nR), eta, qs);
  double* partial = ar.take<double>(RED_BLOCKS);
  double* scal = ar.take<double>(8);  // th2, kept, inv sqrt(kept), r2, norm L, kept (CBE)
  double* stats_local = ar.take<double>(4);
  size_t simt_elems = std::max(gemm_simt_scratch_elems((int)mL, eta, (int)nR, 1),
                               gemm_simt_scratch_elems((int)nR, eta, (int)mL, 1));
  simt_elems = std::max(simt_elems, gemm_simt_scratch_elems(chiL, (int)(d * nR), chiL, 1));
  // block-reflector contractions of the QR (kb x n with K = m, and smaller)
  for (int kb = 1; kb <= 128; kb *= 2)
    simt_elems = std::max(simt_elems, gemm_simt_scratch_elems(kb, eta, (int)std::max(mL, nR), 1));
  cx<T>* simt_scratch = simt_elems ? ar.take<cx<T>>(simt_elems) : nullptr;
  // CBE: the decomposition of L^dag L. complex128: two-sided FP64 Jacobi on M = Rz Rz^dag;
  // complex64: one-sided FP32 Jacobi on the rows of Rz (M is never formed)
  constexpr bool kOneSided = std::is_same<T, float>::value;
  // complex128: the one-sided FP64 Jacobi whenever a block pair of rows fits shared memory,
  // else the two-sided solver on M = Rz Rz^dag
  const bool sj64 = !kOneSided && cbe && svd64_supported(eta);
  double2* M = nullptr; double2* Vh = nullptr; double* w = nullptr; double2* eig_scr = nullptr;
  double* Sv = nullptr; cx<T>* Vt = nullptr; int* chi_dev = nullptr; char* sj_work = nullptr;
  cx<T>* Bn_full = nullptr; cx<T>* Bm_full = nullptr;
  size_t eig_elems = 0, sj_bytes = 0;
  if (cbe) {
    Vh = ar.take<double2>((size_t)eta * eta);
    w = ar.take<double>(eta);
    Sv = ar.take<double>(eta);
    Vt = ar.take<cx<T>>((size_t)eta * eta);
    chi_dev = ar.take<int>(4);
    // the last products run at the expansion eta (rows of V beyond chi~ zeroed) into these,
    // and their first chi~ rows / columns are copied into the outputs' layout
    Bn_full = ar.take<cx<T>>((size_t)eta * nR);
    Bm_full = ar.take<cx<T>>((size_t)mL * eta);
    if (kOneSided || sj64) {
      sj_bytes = kOneSided ? svd32_work_bytes(eta) : svd64_work_bytes(eta);
      sj_work = ar.take<char>(sj_bytes);
    } else {
      M = ar.take<double2>((size_t)eta * eta);
      eig_elems = herm_eig_scratch_elems(eta);
      eig_scr = ar.take<double2>(eig_elems);
    }
  }
  const bool eps_explicit = tr->eps_explicit != 0;
  // one re-orthogonalisation pass of Qz (auto: complex64 with 1xTF32 contractions, whose
  // QR leaves the isometry at the TF32 level; after 3xTF32 it is already at the FP32 floor
  // that the pass's own Gram matrix resolves)
  const bool reorth = tr->reorth > 0 || (tr->reorth < 0 && io->precision == QRTEBD_C64_TF32);
  cx<T>* Dm = reorth ? ar.take<cx<T>>((size_t)eta * eta) : nullptr;
  cx<T>* Qr = reorth ? ar.take<cx<T>>((size_t)nR * eta) : nullptr;
  cx<T>* Rbuf = eps_explicit ? ar.take<cx<T>>((size_t)mL * nR) : nullptr;
  cx<T>* Zc = (eps_explicit && !cbe) ? ar.take<cx<T>>((size_t)nR * eta) : nullptr;
  cx<T>* LV = (eps_explicit && cbe) ? ar.take<cx<T>>((size_t)eta * eta) : nullptr;
  cx<T>* Yt = (eps_explicit && cbe) ? ar.take<cx<T>>((size_t)eta * nR) : nullptr;
  TcWorkspace tcw, tcw_side;
  if (use_tc) tc_carve(ar, (int)std::max(mL, nR), (int)std::max(mL, nR), eta, tcw);
  // the QR's look-ahead updates run on a side stream with their own workspaces
  if (use_tc) tc_carve(ar, (int)std::max(mL, nR), (int)std::max(mL, nR), eta, tcw_side);
  // complex128 on the tensor cores: slices of the larger and the smaller operand of every
  // product (theta' = B^m B^n, when formed, is the widest: both of its sides are large)
  const bool use_oz = std::is_same<T, double>::value && io->precision == QRTEBD_C128_OZ;
  OzWorkspace ozw, ozw_side;
  if (use_oz) {
    const int mx = (int)std::max(mL, nR);
    const int nmax = theta_given ? std::max(eta, chiL) : std::max<int>(eta, (int)std::min(mL, nR));
    oz_carve(ar, mx, mx, nmax, ozw);
    oz_carve(ar, mx, mx, eta, ozw_side);
  }
  cx<T>* simt_scratch_side = simt_elems ? ar.take<cx<T>>(simt_elems) : nullptr;

  if (measuring) { *bytes = ar.off; return QRTEBD_OK; }
  if (ar.overflow()) {
    set_last_message("bond_update: workspace too small");
    return QRTEBD_ERR_OOM;
  }
  unsigned* err = device_error_word();
  GemmRunner<T> runner{io->precision, use_tc ? &tcw : nullptr, simt_scratch, simt_elems, use_oz ? &ozw : nullptr};
  QrGemm<T> qg{qr_gemm_thunk<T>, &runner};
  GemmRunner<T> runner_side{io->precision, use_tc ? &tcw_side : nullptr, simt_scratch_side, simt_elems,
                            use_oz ? &ozw_side : nullptr};
  QrGemm<T> qg_side{qr_gemm_thunk<T>, &runner_side};
  const cx<T> one = mk<T>(1, 0), zero = mk<T>(0, 0);

  // (i) theta' = B^m B^n
  const cx<T>* th = static_cast<const cx<T>*>(io->theta);
  if (!theta_given) {
    GemmArgs<T> g{(int)mL, (int)nR, chiM, static_cast<const cx<T>*>(io->bm), chiM, 1, false,
                  static_cast<const cx<T>*>(io->bn), nR, 1, false, theta_p, nR, 1, one, zero};
    QR_TRY(runner.run(g, st, true));
    th = theta_p;
  }
  // (i) gate (and diagonal Xi)
  const double2* U = static_cast<const double2*>(io->gate);
  const cx<T>* xi = static_cast<const cx<T>*>(io->xi);
  if (theta_gated) {
    if (io->xi_kind == 2) {
      long long tot = mL * nR;
      k_scale_rows<T><<<(unsigned)ceil_div(tot, 256), 256, 0, st>>>(theta_tp, theta_t, xi, chiL,
                                                                   d * nR);
      note_launch();
      QR_CUDA_TRY(cudaGetLastError());
    }
  } else if (d <= 5) {
    QR_TRY(launch_gate<T>(th, theta_tp, U, chiL, d, chiR, io->xi_kind == 2 ? xi : nullptr,
                          io->xi_kind == 2 ? theta_t : nullptr, st));
  } else {
    int n4 = d * d * d * d;
    k_convert_gate<T><<<(unsigned)ceil_div(n4, 256), 256, 0, st>>>(U, Ut, n4);
    note_launch();
    QR_CUDA_TRY(cudaGetLastError());
    GemmArgs<T> g{d * d, chiR, d * d, Ut, d * d, 1, false, th, chiR, 1, false, theta_tp, chiR, 1,
                  one, zero};
    g.batch = chiL; g.bsa = 0; g.bsb = (long long)d * d * chiR; g.bsc = g.bsb;
    QR_TRY(gemm_simt<T>(g, st, nullptr, 0));
    if (io->xi_kind == 2) {
      long long tot = mL * nR;
      k_scale_rows<T><<<(unsigned)ceil_div(tot, 256), 256, 0, st>>>(theta_tp, theta_t, xi, chiL,
                                                                   d * nR);
      note_launch();
      QR_CUDA_TRY(cudaGetLastError());
    }
  }
  if (io->xi_kind == 1 || io->xi_kind == 3) {  // dense Xi: theta~ = Xi theta~' on the left bond index
    GemmArgs<T> g{chiL, (int)(d * nR), chiL, xi, chiL, 1, false, theta_tp, d * nR, 1, false,
                  theta_t, d * nR, 1, one, zero};
    g.tri_a = io->xi_kind == 3;  // lower triangular: blocks above the diagonal are skipped
    QR_TRY(runner.run(g, st, true));
  }
  QR_TRY(norm2<T>(theta_t, mL * nR, partial, scal + 0, st));

  // (i) X = theta~ Y0^dag, QR(X) -> Q
  const cx<T>* Y0 = y0_is_bn ? static_cast<const cx<T>*>(io->bn) : theta_t;
  {
    GemmArgs<T> g{(int)mL, eta, (int)nR, theta_t, nR, 1, false, Y0, 1, nR, true, X, eta, 1, one,
                  zero};
    g.reuse_a = true;  // theta~ is read again, unchanged, by the last contraction
    QR_TRY(runner.run(g, st, true));
  }
  QR_TRY(householder_qr<T>(X, eta, (int)mL, eta, Q, eta, qs, st, err, &qg, &qg_side));

  // (ii) Z = theta~^dag Q, QR(Z) -> Qz, Rz
  {
    GemmArgs<T> g{(int)nR, eta, (int)mL, theta_t, 1, nR, true, Q, eta, 1, false, Z, eta, 1, one,
                  zero};
    QR_TRY(runner.run(g, st, true));
  }
  if (Zc) QR_CUDA_TRY(cudaMemcpyAsync(Zc, Z, (size_t)nR * eta * sizeof(cx<T>), cudaMemcpyDeviceToDevice, st));
  QR_TRY(householder_qr<T>(Z, eta, (int)nR, eta, Qz, eta, qs, st, err, &qg, &qg_side));

  // further sweeps of the alternating least-squares solver (Sec. II comments): the isometry
  // Q^[n] = Qz^dag of the last sweep is kept, X = theta~ Q^[n]^dag = theta~ Qz is the optimal
  // left factor for it, its QR gauges it, and Y = Q^dag theta~ (as Z = theta~^dag Q) is
  // factored again
  for (int sweep = 1; sweep < tr->sweeps; ++sweep) {
    {
      GemmArgs<T> g{(int)mL, eta, (int)nR, theta_t, nR, 1, false, Qz, eta, 1, false, X, eta, 1, one, zero};
      g.reuse_a = true;
      QR_TRY(runner.run(g, st, true));
    }
    QR_TRY(householder_qr<T>(X, eta, (int)mL, eta, Q, eta, qs, st, err, &qg, &qg_side));
    {
      GemmArgs<T> g{(int)nR, eta, (int)mL, theta_t, 1, nR, true, Q, eta, 1, false, Z, eta, 1, one, zero};
      QR_TRY(runner.run(g, st, true));
    }
    if (Zc) QR_CUDA_TRY(cudaMemcpyAsync(Zc, Z, (size_t)nR * eta * sizeof(cx<T>), cudaMemcpyDeviceToDevice, st));
    QR_TRY(householder_qr<T>(Z, eta, (int)nR, eta, Qz, eta, qs, st, err, &qg, &qg_side));
  }

  // the re-orthogonalisation passes run in 3xTF32 whatever the precision
  const GemmRunner<T> runner3{use_tc ? (int)QRTEBD_C64_3XTF32 : io->precision, runner.tc,
                              runner.simt_scratch, runner.simt_scratch_elems};
  if (reorth) {
    // One re-orthogonalisation pass of the right isometry (precision pattern (1)): with
    // D = Qz^dag Qz - 1, Qz <- Qz (1 - D/2), the first-order polar (Newton-Schulz) step,
    // which leaves ||Qz^dag Qz - 1|| at O(||D||^2) plus the storage rounding. Both
    // contractions run in 3xTF32 with FP32 accumulation whatever the precision, so that
    // D is resolved well below the TF32 rounding it corrects; D is formed in the epilogue
    // (beta = 1 onto -1) and the update is added onto a copy of Qz, so neither result is
    // swamped by the O(1) parts.
    k_scaled_eye<T><<<(unsigned)ceil_div((long long)eta * eta, 256), 256, 0, st>>>(Dm, eta, T(-1));
    note_launch();
    QR_CUDA_TRY(cudaGetLastError());
    GemmArgs<T> gd{eta, eta, (int)nR, Qz, 1, eta, true, Qz, eta, 1, false, Dm, eta, 1, one, one};
    QR_TRY(runner3.run(gd, st, true));
    QR_CUDA_TRY(cudaMemcpyAsync(Qr, Qz, (size_t)nR * eta * sizeof(cx<T>), cudaMemcpyDeviceToDevice, st));
    GemmArgs<T> gu{(int)nR, eta, eta, Qz, eta, 1, false, Dm, eta, 1, false, Qr, eta, 1,
                   mk<T>(-0.5, 0), one};
    QR_TRY(runner3.run(gu, st, true));
    std::swap(Qz, Qr);
  }

  cx<T>* bn_out = static_cast<cx<T>*>(io->bn_out);
  cx<T>* xi_out = static_cast<cx<T>*>(io->xi_out);
  cx<T>* bm_out = static_cast<cx<T>*>(io->bm_out);
  int chi_new = eta;
  if (!cbe) {
    // (iii) Xi~ = L / ||L||, B~^n = Q^[n] = Qz^dag, B~^m = theta~' Qz
    QR_TRY(norm2<T>(Z, (long long)eta * eta, partial, scal + 1, st));
    k_finalize<<<1, 1, 0, st>>>(scal + 0, scal + 1, (double)eta,
                                io->stats_out ? io->stats_out : stats_local, scal + 2, err);
    note_launch();
    QR_CUDA_TRY(cudaGetLastError());
    QR_TRY(conj_transpose<T>(Z, eta, xi_out, eta, eta, eta, scal + 2, st));
    QR_TRY(conj_transpose<T>(Qz, eta, bn_out, nR, (int)nR, eta, nullptr, st));
    GemmArgs<T> g{(int)mL, eta, (int)nR, theta_tp, nR, 1, false, Qz, eta, 1, false, bm_out, eta,
                  1, one, zero};
    g.reuse_a = true;
    QR_TRY(runner.run(g, st, true));
    if (eps_explicit) {
      // residual theta~ - Q Y with Y = Zc^dag (Sec. IV: the explicit distance)
      QR_CUDA_TRY(cudaMemcpyAsync(Rbuf, theta_t, (size_t)mL * nR * sizeof(cx<T>), cudaMemcpyDeviceToDevice, st));
      GemmArgs<T> r{(int)mL, (int)nR, eta, Q, eta, 1, false, Zc, 1, eta, true, Rbuf, nR, 1,
                    mk<T>(-1, 0), one};
      QR_TRY(runner.run(r, st, true));
      QR_TRY(norm2<T>(Rbuf, mL * nR, partial, scal + 3, st));
      k_eps_explicit<<<1, 1, 0, st>>>(scal + 0, scal + 3, io->stats_out ? io->stats_out : stats_local);
      note_launch();
      QR_CUDA_TRY(cudaGetLastError());
    }
  } else {
    // (iv) L^dag L = Rz Rz^dag = V^dag S^2 V: w = S^2 descending, Vh = V (rows)
    long long ee = (long long)eta * eta;
    QR_TRY(norm2<T>(Z, ee, partial, scal + 4, st));  // ||L||^2 in FP64
    if constexpr (kOneSided) {
      QR_TRY(svd_rows_jacobi32(reinterpret_cast<const float2*>(Z), eta, eta, w, Vh, sj_work, sj_bytes,
                               st, err));
    } else if (sj64) {
      QR_TRY(svd_rows_jacobi64(reinterpret_cast<const double2*>(Z), eta, eta, w, Vh, sj_work, sj_bytes,
                               st, err));
    } else {
      double2* Rz64 = M;  // reuse: first convert Rz, then form M in Vh's buffer, swap
      k_to_c128<T><<<(unsigned)ceil_div(ee, 256), 256, 0, st>>>(Z, Rz64, ee);
      note_launch();
      QR_CUDA_TRY(cudaGetLastError());
      {
        GemmArgs<double> g{eta, eta, eta, Rz64, eta, 1, false, Rz64, 1, eta, true, Vh, eta, 1,
                           mk<double>(1, 0), mk<double>(0, 0)};
        QR_TRY(gemm_simt<double>(g, st, nullptr, 0));
      }
      // Vh now holds M; eig destroys its input -> copy into M and decompose
      QR_CUDA_TRY(cudaMemcpyAsync(M, Vh, ee * sizeof(double2), cudaMemcpyDeviceToDevice, st));
      QR_TRY(herm_eig(M, eta, w, Vh, eig_scr, eig_elems, st, err));
    }
    k_cbe_cut<<<1, 1, 0, st>>>(w, eta, tr->chi_max, tr->svd_min, tr->tie_tol, tr->eps_target, scal + 4,
                               Sv, scal + 1, scal + 5, chi_dev);
    note_launch();
    QR_CUDA_TRY(cudaGetLastError());
    if (io->schmidt_out)
      QR_CUDA_TRY(cudaMemcpyAsync(io->schmidt_out, Sv, eta * sizeof(double), cudaMemcpyDeviceToDevice, st));
    k_finalize<<<1, 1, 0, st>>>(scal + 0, scal + 1, 0.0, io->stats_out ? io->stats_out : stats_local, scal + 2,
                                err, scal + 5, chi_dev);
    note_launch();
    QR_CUDA_TRY(cudaGetLastError());
    // (v) with chi~ on the device: Vt = P V (rows from chi~ on zeroed), B~^n = P V Q^[n] at
    // eta rows (Bn_full = Vt Qz^dag), Xi~ = diag(S[0:chi~]) / ||.||, B~^m = theta~' B~^n^dag at
    // eta columns; the outputs take the first chi~ rows / columns
    const unsigned gb = (unsigned)ceil_div(ee, 256);
    k_from_c128_rows<T><<<gb, 256, 0, st>>>(Vh, Vt, eta, chi_dev);
    note_launch();
    QR_CUDA_TRY(cudaGetLastError());
    {
      GemmArgs<T> g{eta, (int)nR, eta, Vt, eta, 1, false, Qz, 1, eta, true, Bn_full, nR, 1, one, zero};
      QR_TRY(runner.run(g, st, true));
    }
    k_copy_rows_dev<T><<<(unsigned)ceil_div((long long)eta * nR, 256), 256, 0, st>>>(Bn_full, bn_out, nR, eta, chi_dev);
    note_launch();
    k_diag_xi_dev<T><<<gb, 256, 0, st>>>(Sv, chi_dev, eta, scal + 2, xi_out);
    note_launch();
    QR_CUDA_TRY(cudaGetLastError());
    {
      GemmArgs<T> g{(int)mL, eta, (int)nR, theta_tp, nR, 1, false, Bn_full, 1, nR, true, Bm_full, eta, 1,
                    one, zero};
      QR_TRY(runner.run(g, st, true));
    }
    k_copy_cols_dev<T><<<(unsigned)ceil_div((long long)mL * eta, 256), 256, 0, st>>>(Bm_full, eta, bm_out, mL, chi_dev);
    note_launch();
    QR_CUDA_TRY(cudaGetLastError());
    if (eps_explicit) {
      // approx = Q L V_c^dag B~^n = Q (L Vt^dag) Bn_full; residual theta~ - approx (Sec. IV)
      GemmArgs<T> g1{eta, eta, eta, Z, 1, eta, true, Vt, 1, eta, true, LV, eta, 1, one, zero};
      QR_TRY(runner.run(g1, st));
      GemmArgs<T> g2{eta, (int)nR, eta, LV, eta, 1, false, Bn_full, nR, 1, false, Yt, nR, 1, one, zero};
      QR_TRY(runner.run(g2, st));
      QR_CUDA_TRY(cudaMemcpyAsync(Rbuf, theta_t, (size_t)mL * nR * sizeof(cx<T>), cudaMemcpyDeviceToDevice, st));
      GemmArgs<T> r{(int)mL, (int)nR, eta, Q, eta, 1, false, Yt, nR, 1, false, Rbuf, nR, 1,
                    mk<T>(-1, 0), one};
      QR_TRY(runner.run(r, st, true));
      QR_TRY(norm2<T>(Rbuf, mL * nR, partial, scal + 3, st));
      k_eps_explicit<<<1, 1, 0, st>>>(scal + 0, scal + 3, io->stats_out ? io->stats_out : stats_local);
      note_launch();
      QR_CUDA_TRY(cudaGetLastError());
    }
    chi_new = -1;
    if (sync_chi) {
      int chi_h = 0;
      QR_CUDA_TRY(cudaMemcpyAsync(&chi_h, chi_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
      QR_CUDA_TRY(cudaStreamSynchronize(st));
      if (chi_h < 1 || chi_h > eta) { set_last_message("CBE: bad cut"); return QRTEBD_ERR_NUMERIC; }
      chi_new = chi_h;
    }
  }
  if (info) { info->eta = eta; info->chi_new = chi_new; }
  return QRTEBD_OK;
}

}  // namespace

int choose_eta(const qrtebd_trunc* tr, int chi_l, int d, int chi_m, int chi_r) {
  long long cap = std::min((long long)d * chi_l, (long long)d * chi_r);
  long long eta;
  if (tr->eta > 0) {
    eta = tr->eta;
  } else if (tr->scheme == QRTEBD_PLAIN) {
    eta = std::min<long long>(tr->chi_max, cap);
  } else {
    long long dchi = (long long)std::ceil(tr->dchi_frac * chi_m - 1e-9);
    if (dchi < tr->dchi_min) dchi = tr->dchi_min;
    eta = std::min<long long>(chi_m + dchi, cap);
  }
  if (eta < 1 || eta > cap) return -1;
  return (int)eta;
}

int bond_update(const qrtebd_bond_io* io, const qrtebd_trunc* tr, cudaStream_t st,
                qrtebd_bond_info* info, size_t* bytes, bool sync_chi, bool theta_gated) {
  if (!io || !tr) return QRTEBD_ERR_INVALID_ARG;
  if (theta_gated && !bytes && !io->theta) return QRTEBD_ERR_INVALID_ARG;
  if (io->chi_l < 1 || io->d < (theta_gated ? 1 : 2) || io->chi_m < 1 || io->chi_r < 1 || tr->chi_max < 1)
    return QRTEBD_ERR_INVALID_ARG;
  if (io->xi_kind < 0 || io->xi_kind > 3) return QRTEBD_ERR_INVALID_ARG;
  if (tr->scheme != QRTEBD_PLAIN && tr->scheme != QRTEBD_CBE) return QRTEBD_ERR_INVALID_ARG;
  if (tr->sweeps < 0 || tr->sweeps > 1000) {
    set_last_message("bond_update: sweeps must lie in 0..1000");
    return QRTEBD_ERR_INVALID_ARG;
  }
  if (!bytes) {
    if (!io->bn || (!io->gate && !theta_gated) || !io->bm_out || !io->xi_out || !io->bn_out) return QRTEBD_ERR_INVALID_ARG;
    if (!io->theta && !io->bm) return QRTEBD_ERR_INVALID_ARG;
    if (io->xi_kind != 0 && !io->xi) return QRTEBD_ERR_INVALID_ARG;
  }
  switch (io->precision) {
    case QRTEBD_C128:
    case QRTEBD_C128_OZ: return bond_update_t<double>(io, tr, st, info, bytes, sync_chi, theta_gated);
    case QRTEBD_C64_3XTF32:
    case QRTEBD_C64_TF32:
    case QRTEBD_C64_FP32: return bond_update_t<float>(io, tr, st, info, bytes, sync_chi, theta_gated);
    default: return QRTEBD_ERR_INVALID_ARG;
  }
}

}  // namespace qrtebd
