// CBE with Z_d charge sectors (Sec. III, closing paragraphs); see qrtebd.h.
//
// With a global Z_d symmetry theta~ (a (chi_l d) x (d chi_r) matrix) is block diagonal up to
// a permutation: block q holds the rows alpha*d + i with c_l(alpha) + i = q and the columns
// j*chi_r + delta with c_r(delta) - j = q. Steps (i)-(iv) of CBE then run block by block:
//   1. k_sym_gather: theta~'_q = U theta' for the entries of every block, read straight from
//      the dense theta' (only the entries the charge rule allows are touched; the gate keeps
//      i + j mod d, so each output sums d products instead of d^2);
//   2. per block, concurrently, the dense CBE update (bond_update with the gate applied, d = 1,
//      eta_q = min(chi_q + dchi_q, rows_q, cols_q), every Schmidt value kept);
//   3. k_sym_cut: one cut over the Schmidt values of all blocks (merged by rank, the dense
//      rule of qrtebd_trunc), giving chi~ and each block's share chi~_q on the device;
//   4. k_sym_scatter_*: the first chi~_q states of every block into the dense outputs, block
//      by block in increasing charge; Xi~ = diag(S) / ||kept||.
// The blocks of step 2 run concurrently on library-owned streams. One stream synchronisation
// at the end returns chi~_q to the host (for the charge labels).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "bond.cuh"

namespace qrtebd {

namespace {

constexpr int kSymMaxD = 16;

// host plan: the blocks' sizes, the maps between dense rows/columns and block positions,
// and where each block's data sits in the workspace
struct SymMeta {
  int d, nsec, chiR;
  int nrow[kSymMaxD], ncol[kSymMaxD], eta[kSymMaxD];
  long long row_off[kSymMaxD + 1], col_off[kSymMaxD + 1];  // into rowmap / colmap
  long long el_off[kSymMaxD + 1];                          // theta~'_q blocks (elements)
  long long bm_off[kSymMaxD + 1], bn_off[kSymMaxD + 1], xi_off[kSymMaxD + 1];
  long long s_off[kSymMaxD + 1];                           // Schmidt values (eta_q each)
};

struct SymPlan {
  SymMeta m;
  int chi_q[kSymMaxD];
  int eta_sum = 0;
  std::vector<int> ints;  // rowmap | colmap | rowsec | rowpos | colsec | colpos
  long long nrows = 0, ncols = 0;
};

int make_plan(const qrtebd_sym_bond_io* io, const qrtebd_trunc* tr, SymPlan& p) {
  const int d = io->d, chiL = io->chi_l, chiR = io->chi_r, chiM = io->chi_m;
  if (d < 2 || d > kSymMaxD) {
    set_last_message("sym_bond_update: d must lie in 2..16");
    return QRTEBD_ERR_INVALID_ARG;
  }
  if (chiL < 1 || chiM < 1 || chiR < 1 || tr->chi_max < 1) return QRTEBD_ERR_INVALID_ARG;
  if (!io->charge_l || !io->charge_m || !io->charge_r) return QRTEBD_ERR_INVALID_ARG;
  if (tr->scheme != QRTEBD_CBE || tr->eta != 0) {
    set_last_message("sym_bond_update: needs scheme CBE with eta = 0 (eta is set per block)");
    return QRTEBD_ERR_INVALID_ARG;
  }
  if (io->xi_kind != 0 && io->xi_kind != 2) {
    set_last_message("sym_bond_update: Xi must be the identity or diagonal");
    return QRTEBD_ERR_INVALID_ARG;
  }
  auto valid = [d](const int* c, int n) {
    for (int k = 0; k < n; ++k) if (c[k] < 0 || c[k] >= d) return false;
    return true;
  };
  if (!valid(io->charge_l, chiL) || !valid(io->charge_m, chiM) || !valid(io->charge_r, chiR)) {
    set_last_message("sym_bond_update: charges must lie in 0..d-1");
    return QRTEBD_ERR_INVALID_ARG;
  }
  SymMeta& m = p.m;
  std::memset(&m, 0, sizeof m);
  m.d = d; m.nsec = d; m.chiR = chiR;
  p.nrows = (long long)chiL * d;
  p.ncols = (long long)d * chiR;
  std::vector<std::vector<int>> rows(d), cols(d);
  for (int a = 0; a < chiL; ++a)
    for (int i = 0; i < d; ++i) rows[(io->charge_l[a] + i) % d].push_back(a * d + i);
  for (int j = 0; j < d; ++j)
    for (int b = 0; b < chiR; ++b) cols[((io->charge_r[b] - j) % d + d) % d].push_back(j * chiR + b);
  for (int q = 0; q < d; ++q) p.chi_q[q] = 0;
  for (int g = 0; g < chiM; ++g) p.chi_q[io->charge_m[g]]++;
  p.ints.assign((size_t)(3 * p.nrows + 3 * p.ncols), 0);
  int* rowmap = p.ints.data();
  int* colmap = rowmap + p.nrows;
  int* rowsec = colmap + p.ncols;
  int* rowpos = rowsec + p.nrows;
  int* colsec = rowpos + p.nrows;
  int* colpos = colsec + p.ncols;
  p.eta_sum = 0;
  for (int q = 0; q < d; ++q) {
    const int nr = (int)rows[q].size(), nc = (int)cols[q].size();
    m.nrow[q] = nr; m.ncol[q] = nc;
    int eta = 0;
    if (nr > 0 && nc > 0) {
      long long dchi = (long long)std::ceil(tr->dchi_frac * p.chi_q[q] - 1e-9);
      if (dchi < tr->dchi_min) dchi = tr->dchi_min;
      eta = (int)std::min<long long>({(long long)p.chi_q[q] + dchi, (long long)nr, (long long)nc});
    }
    m.eta[q] = eta;
    p.eta_sum += eta;
    m.row_off[q + 1] = m.row_off[q] + nr;
    m.col_off[q + 1] = m.col_off[q] + nc;
    m.el_off[q + 1] = m.el_off[q] + (long long)nr * nc;
    m.bm_off[q + 1] = m.bm_off[q] + (long long)nr * eta;
    m.bn_off[q + 1] = m.bn_off[q] + (long long)eta * nc;
    m.xi_off[q + 1] = m.xi_off[q] + (long long)eta * eta;
    m.s_off[q + 1] = m.s_off[q] + eta;
    for (int k = 0; k < nr; ++k) {
      rowmap[m.row_off[q] + k] = rows[q][k];
      rowsec[rows[q][k]] = q;
      rowpos[rows[q][k]] = k;
    }
    for (int k = 0; k < nc; ++k) {
      colmap[m.col_off[q] + k] = cols[q][k];
      colsec[cols[q][k]] = q;
      colpos[cols[q][k]] = k;
    }
  }
  if (p.eta_sum < 1) {
    set_last_message("sym_bond_update: no block has both rows and columns");
    return QRTEBD_ERR_INVALID_ARG;
  }
  return QRTEBD_OK;
}

// The blocks run concurrently, each on a library-owned stream forked from the caller's and
// joined back to it (one set per device and caller stream, as the QR's side streams).
struct BlockStreams {
  cudaStream_t st[kSymMaxD] = {};
  cudaEvent_t fork = nullptr;
  cudaEvent_t done[kSymMaxD] = {};
};
std::mutex g_blk_mu;
std::map<std::pair<int, cudaStream_t>, BlockStreams> g_blk;

int block_streams(cudaStream_t main, BlockStreams** out) {
  int dev = 0;
  QR_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_blk_mu);
  BlockStreams& b = g_blk[std::make_pair(dev, main)];
  if (!b.fork) {
    for (int q = 0; q < kSymMaxD; ++q) {
      QR_CUDA_TRY(cudaStreamCreateWithFlags(&b.st[q], cudaStreamNonBlocking));
      QR_CUDA_TRY(cudaEventCreateWithFlags(&b.done[q], cudaEventDisableTiming));
    }
    QR_CUDA_TRY(cudaEventCreateWithFlags(&b.fork, cudaEventDisableTiming));
  }
  *out = &b;
  return QRTEBD_OK;
}

// the dense CBE update of block q (gate applied, d = 1, every Schmidt value kept)
void block_io(const qrtebd_sym_bond_io* io, const SymPlan& p, int q, qrtebd_bond_io& b,
              qrtebd_trunc& t, const qrtebd_trunc* tr) {
  std::memset(&b, 0, sizeof b);
  b.precision = io->precision;
  b.chi_l = p.m.nrow[q];
  b.d = 1;
  b.chi_m = std::max(1, p.chi_q[q]);
  b.chi_r = p.m.ncol[q];
  b.xi_kind = io->xi_kind;
  t = *tr;
  t.scheme = QRTEBD_CBE;
  t.chi_max = p.m.eta[q];
  t.eta = p.m.eta[q];
  t.svd_min = 0.0;
  t.tie_tol = 0.0;
  t.eps_target = 0.0;
  t.eps_explicit = 0;
}

// ------------------------------------------------------------------ kernels
// theta~'_q[r, c] = sum_{i'} U[(i j), (i' j')] theta'[alpha, i', j', delta], j' = i + j - i'
// (mod d), for every element of every block; (alpha, i) and (j, delta) from the maps
template <typename T>
__global__ void k_sym_gather(const cx<T>* __restrict__ th, const double2* __restrict__ U,
                             cx<T>* __restrict__ out, const int* __restrict__ rowmap,
                             const int* __restrict__ colmap, SymMeta m) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= m.el_off[m.nsec]) return;
  int q = 0;
  while (q + 1 < m.nsec && idx >= m.el_off[q + 1]) ++q;
  const long long loc = idx - m.el_off[q];
  const int nc = m.ncol[q];
  const int r = (int)(loc / nc), c = (int)(loc % nc);
  const int d = m.d;
  const int gr = rowmap[m.row_off[q] + r], gc = colmap[m.col_off[q] + c];
  const int a = gr / d, i = gr % d, j = gc / m.chiR, delta = gc % m.chiR;
  const int t = (i + j) % d;
  const long long d2 = (long long)d * d;
  const double2* Urow = U + (long long)(i * d + j) * d2;
  const cx<T>* tha = th + (long long)a * d2 * m.chiR + delta;
  cx<T> acc = mk<T>(0, 0);
  for (int ip = 0; ip < d; ++ip) {
    const int jp = (t - ip + d) % d;
    const double2 u = __ldg(Urow + ip * d + jp);
    cfma<T>(acc, mk<T>((T)u.x, (T)u.y), tha[(long long)(ip * d + jp) * m.chiR]);
  }
  out[idx] = acc;
}

// the diagonal of Xi per row of every block: rowxi[k] = xi[alpha(rowmap[k])]
template <typename T>
__global__ void k_sym_rowxi(const cx<T>* __restrict__ xi, const int* __restrict__ rowmap,
                            cx<T>* __restrict__ rowxi, long long n, int d) {
  const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k < n) rowxi[k] = xi[rowmap[k] / d];
}

struct SymCutArgs {
  const double* S;      // Schmidt values, block q at s_off[q], descending
  const double* stats;  // per block: eps, ||theta~_q||^2, ||L_q||^2 (all kept), chi_q kept
  double* merged;       // eta_sum: all values in merged order
  int* out;             // [0, d): chi~_q; [d, 2d+1): offsets; [2d+1, 3d+1): block strides
  double* scal;         // [0]: 1 / ||kept||
  double* stats_out;    // eps, ||theta~||^2, kept, chi~ (optional)
  unsigned* err;
  int chi_max;
  double svd_min, tie_tol, eps_target;
};

// number of values of block qq (descending, n of them) that come before value v of block q in
// the merged order: larger values, and equal ones of a lower charge
__device__ int count_before(const double* s, int n, double v, bool lower_charge) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    const bool before = lower_charge ? (s[mid] >= v) : (s[mid] > v);
    if (before) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// One cut over all blocks (one CTA): every value's rank in the merged order from binary
// searches in the other blocks, the dense cut rule on the merged list (thread 0, in order),
// and each block's share chi~_q = the number of its values ranked below chi~.
__global__ void k_sym_cut(SymMeta m, SymCutArgs a) {
  __shared__ int cnt[kSymMaxD];
  __shared__ int c_sh;
  __shared__ int bad;
  const int d = m.nsec;
  if (threadIdx.x < kSymMaxD) cnt[threadIdx.x] = 0;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  const int n = (int)m.s_off[d];
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    int q = 0;
    while (q + 1 < d && t >= m.s_off[q + 1]) ++q;
    const int k = t - (int)m.s_off[q];
    const double v = a.S[t];
    if (!(v >= 0.0) || !isfinite(v)) { bad = 1; continue; }
    int rank = k;
    for (int qq = 0; qq < d; ++qq)
      if (qq != q) rank += count_before(a.S + m.s_off[qq], m.eta[qq], v, qq < q);
    a.merged[rank < n ? rank : n - 1] = v;
  }
  __syncthreads();
  if (bad) {
    if (threadIdx.x == 0) atomicOr(a.err, DEVERR_NUMERIC);
  }
  if (threadIdx.x == 0) {
    double tot = 0.0, th2 = 0.0;
    for (int q = 0; q < d; ++q) { tot += a.stats[4 * q + 2]; th2 += a.stats[4 * q + 1]; }
    if (!(tot > 0)) { tot = 0; for (int k = 0; k < n; ++k) tot += a.merged[k] * a.merged[k]; }
    const double nrm = sqrt(tot);
    int c = 0;
    if (nrm > 0) { while (c < n && a.merged[c] / nrm >= a.svd_min) ++c; }
    if (c > a.chi_max) c = a.chi_max;
    if (c < 1) c = 1;
    if (a.eps_target > 0 && tot > 0) {
      double tail = 0;
      int ce = n;
      while (ce > 1 && tail + a.merged[ce - 1] * a.merged[ce - 1] <= a.eps_target * tot) {
        tail += a.merged[ce - 1] * a.merged[ce - 1];
        --ce;
      }
      if (ce < c) c = ce;
    }
    if (nrm > 0) {
      while (c < n && c > 1 && (a.merged[c - 1] - a.merged[c]) / nrm <= a.tie_tol * (a.merged[0] / nrm)) --c;
    }
    if (bad) c = 1;
    c_sh = c;
    (void)th2;
  }
  __syncthreads();
  const int c = c_sh;
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    int q = 0;
    while (q + 1 < d && t >= m.s_off[q + 1]) ++q;
    const int k = t - (int)m.s_off[q];
    const double v = a.S[t];
    if (!(v >= 0.0) || !isfinite(v)) continue;
    int rank = k;
    for (int qq = 0; qq < d; ++qq)
      if (qq != q) rank += count_before(a.S + m.s_off[qq], m.eta[qq], v, qq < q);
    if (rank < c) atomicAdd(&cnt[q], 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0, th2 = 0.0, kk = 0.0, tail = 0.0;
    int off = 0;
    for (int q = 0; q < d; ++q) {
      tot += a.stats[4 * q + 2];
      th2 += a.stats[4 * q + 1];
      const int kept_blk = (int)a.stats[4 * q + 3];  // the block's own outputs hold this many
      int cq = cnt[q];
      if (bad) cq = (off == 0 && m.eta[q] > 0) ? 1 : 0;
      if (cq > kept_blk) cq = kept_blk;
      a.out[q] = cq;
      a.out[d + q] = off;
      a.out[2 * d + 1 + q] = kept_blk;
      off += cq;
      const double* s = a.S + m.s_off[q];
      for (int k = 0; k < cq; ++k) kk += s[k] * s[k];
      for (int k = m.eta[q] - 1; k >= cq; --k) tail += s[k] * s[k];  // smallest first
    }
    a.out[2 * d] = off;
    if (!(tot > 0)) tot = kk + tail;
    const double kept = tot - tail;
    double eps = th2 > 0 ? 1.0 - kept / th2 : 0.0;
    if (eps < 0) eps = 0;
    if (!isfinite(th2) || !isfinite(kept)) atomicOr(a.err, DEVERR_NUMERIC);
    a.scal[0] = kk > 0 ? 1.0 / sqrt(kk) : 0.0;
    if (a.stats_out) {
      a.stats_out[0] = eps;
      a.stats_out[1] = th2;
      a.stats_out[2] = kept;
      a.stats_out[3] = (double)off;
    }
  }
}

__device__ __forceinline__ int sector_of(const int* off, int d, int col) {
  int q = 0;
  while (q + 1 < d && col >= off[q + 1]) ++q;
  return q;
}

// B~^m (chi_l d) x chi~: column col of block q (k = col - off_q) takes block q's column k
// on the rows of block q, zero elsewhere. Grid over rows x cap; columns >= chi~ return.
template <typename T>
__global__ void k_sym_scatter_bm(const cx<T>* __restrict__ bmq, const int* __restrict__ rowsec,
                                 const int* __restrict__ rowpos, const int* __restrict__ out_i,
                                 SymMeta m, cx<T>* __restrict__ bm_out, long long rows, int cap) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= rows * cap) return;
  const int d = m.nsec;
  const int chi = out_i[2 * d];
  const long long r = idx / cap;
  const int col = (int)(idx % cap);
  if (col >= chi) return;
  const int q = sector_of(out_i + d, d, col);
  const int k = col - out_i[d + q];
  const int stride = out_i[2 * d + 1 + q];
  cx<T> v = mk<T>(0, 0);
  if (rowsec[r] == q) v = bmq[m.bm_off[q] + (long long)rowpos[r] * stride + k];
  bm_out[r * chi + col] = v;
}

// B~^n chi~ x (d chi_r): row g of block q takes block q's row k on the columns of block q
template <typename T>
__global__ void k_sym_scatter_bn(const cx<T>* __restrict__ bnq, const int* __restrict__ colsec,
                                 const int* __restrict__ colpos, const int* __restrict__ out_i,
                                 SymMeta m, cx<T>* __restrict__ bn_out, long long cols, int cap) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= cols * cap) return;
  const int d = m.nsec;
  const int chi = out_i[2 * d];
  const int g = (int)(idx / cols);
  const long long c = idx % cols;
  if (g >= chi) return;
  const int q = sector_of(out_i + d, d, g);
  const int k = g - out_i[d + q];
  cx<T> v = mk<T>(0, 0);
  if (colsec[c] == q) v = bnq[m.bn_off[q] + (long long)k * m.ncol[q] + colpos[c]];
  bn_out[(long long)g * cols + c] = v;
}

template <typename T>
__global__ void k_sym_xi(const double* __restrict__ S, const int* __restrict__ out_i, SymMeta m,
                         const double* __restrict__ scal, cx<T>* __restrict__ xi_out, int cap) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  const int d = m.nsec;
  if (g >= cap || g >= out_i[2 * d]) return;
  const int q = sector_of(out_i + d, d, g);
  const int k = g - out_i[d + q];
  xi_out[g] = mk<T>((T)(S[m.s_off[q] + k] * scal[0]), (T)0);
}

template <typename T>
int sym_update_t(const qrtebd_sym_bond_io* io, const qrtebd_trunc* tr, cudaStream_t st,
                 qrtebd_bond_info* info, size_t* bytes, int* eta_sum_out) {
  SymPlan p;
  QR_TRY(make_plan(io, tr, p));
  const SymMeta& m = p.m;
  const int d = io->d;
  if (eta_sum_out) *eta_sum_out = p.eta_sum;
  const int cap = std::min(tr->chi_max, p.eta_sum);
  const bool measuring = (bytes != nullptr);

  // the inner workspace of every block (they run concurrently)
  size_t inner[kSymMaxD] = {};
  for (int q = 0; q < d; ++q) {
    if (m.eta[q] == 0) continue;
    qrtebd_bond_io b;
    qrtebd_trunc t;
    block_io(io, p, q, b, t, tr);
    static const char dummy = 0;
    b.theta = &dummy;
    QR_TRY(bond_update(&b, &t, nullptr, nullptr, &inner[q], true, /*theta_gated=*/true));
  }

  Arena ar;
  ar.measuring = measuring;
  if (!measuring) { ar.base = static_cast<char*>(io->workspace); ar.cap = io->workspace_bytes; }
  int* ints = ar.take<int>(p.ints.size());
  cx<T>* tg = ar.take<cx<T>>((size_t)m.el_off[d]);
  cx<T>* rowxi = io->xi_kind == 2 ? ar.take<cx<T>>((size_t)p.nrows) : nullptr;
  cx<T>* bmq = ar.take<cx<T>>((size_t)m.bm_off[d]);
  cx<T>* bnq = ar.take<cx<T>>((size_t)m.bn_off[d]);
  cx<T>* xiq = ar.take<cx<T>>((size_t)m.xi_off[d]);
  double* S = ar.take<double>((size_t)m.s_off[d]);
  double* stq = ar.take<double>(4 * kSymMaxD);
  double* merged = ar.take<double>((size_t)p.eta_sum);
  double* scal = ar.take<double>(4);
  int* out_i = ar.take<int>(3 * kSymMaxD + 2);
  char* inner_ws[kSymMaxD] = {};
  for (int q = 0; q < d; ++q) inner_ws[q] = inner[q] ? ar.take<char>(inner[q]) : nullptr;
  // theta' = B^m B^n when it is not given (a dense product; the charge rule makes the entries
  // outside the blocks exact zeros)
  const bool theta_given = io->theta != nullptr || (measuring && io->bm == nullptr);
  const long long mL = p.nrows, nR = p.ncols;
  cx<T>* theta_p = theta_given ? nullptr : ar.take<cx<T>>((size_t)(mL * nR));
  const size_t zg_bytes = theta_given ? 0 : qrtebd_zgemm_workspace_size((int)mL, (int)nR, io->chi_m);
  char* zg_ws = theta_given ? nullptr : ar.take<char>(zg_bytes);
  if (measuring) { *bytes = ar.off; return QRTEBD_OK; }
  if (ar.overflow()) {
    set_last_message("sym_bond_update: workspace too small");
    return QRTEBD_ERR_OOM;
  }
  if ((!io->theta && (!io->bm || !io->bn)) || !io->gate || !io->bm_out || !io->xi_out || !io->bn_out || !io->charge_out ||
      (io->xi_kind == 2 && !io->xi))
    return QRTEBD_ERR_INVALID_ARG;
  unsigned* err = device_error_word();
  const int* rowmap = ints;
  const int* colmap = rowmap + p.nrows;
  const int* rowsec = colmap + p.ncols;
  const int* rowpos = rowsec + p.nrows;
  const int* colsec = rowpos + p.nrows;
  const int* colpos = colsec + p.ncols;
  QR_CUDA_TRY(cudaMemcpyAsync(ints, p.ints.data(), p.ints.size() * sizeof(int),
                              cudaMemcpyHostToDevice, st));

  const cx<T>* th = static_cast<const cx<T>*>(io->theta);
  if (!theta_given) {
    const double one[2] = {1, 0}, zero[2] = {0, 0};
    QR_TRY(qrtebd_zgemm(io->precision, (int)mL, (int)nR, io->chi_m, io->bm, io->chi_m, 1, 0, io->bn,
                        nR, 1, 0, theta_p, nR, 1, one, zero, zg_ws, zg_bytes, st));
    th = theta_p;
  }
  // 1. gate and gather every block
  const long long nel = m.el_off[d];
  if (nel > 0) {
    k_sym_gather<T><<<(unsigned)ceil_div(nel, 256), 256, 0, st>>>(
        th, static_cast<const double2*>(io->gate), tg, rowmap,
        colmap, m);
    note_launch();
    QR_CUDA_TRY(cudaGetLastError());
  }
  if (rowxi) {
    k_sym_rowxi<T><<<(unsigned)ceil_div(p.nrows, 256), 256, 0, st>>>(
        static_cast<const cx<T>*>(io->xi), rowmap, rowxi, p.nrows, d);
    note_launch();
    QR_CUDA_TRY(cudaGetLastError());
  }
  // 2. the dense CBE update of every block, all blocks at once on their own streams (a block
  //    alone leaves most of the GPU idle: its panels and Jacobi steps are latency-bound); the
  //    QR inside each forks its own side streams
  QR_CUDA_TRY(cudaMemsetAsync(stq, 0, 4 * kSymMaxD * sizeof(double), st));
  BlockStreams* bs = nullptr;
  QR_TRY(block_streams(st, &bs));
  QR_CUDA_TRY(cudaEventRecord(bs->fork, st));
  int rc = QRTEBD_OK;
  int nblk = 0;
  for (int q = 0; q < d; ++q) nblk += m.eta[q] > 0;
  ConcurrencyScope conc(nblk);
  for (int q = 0; q < d; ++q) {
    if (m.eta[q] == 0) continue;
    QR_CUDA_TRY(cudaStreamWaitEvent(bs->st[q], bs->fork, 0));
    qrtebd_bond_io b;
    qrtebd_trunc t;
    block_io(io, p, q, b, t, tr);
    b.theta = tg + m.el_off[q];
    b.bn = tg + m.el_off[q];  // not read: CBE takes Y0 from theta~
    b.xi = rowxi ? rowxi + m.row_off[q] : nullptr;
    b.bm_out = bmq + m.bm_off[q];
    b.bn_out = bnq + m.bn_off[q];
    b.xi_out = xiq + m.xi_off[q];
    b.stats_out = stq + 4 * q;
    b.schmidt_out = S + m.s_off[q];
    b.workspace = inner_ws[q];
    b.workspace_bytes = inner[q];
    qrtebd_bond_info bi;
    if (rc == QRTEBD_OK)
      rc = bond_update(&b, &t, bs->st[q], &bi, nullptr, /*sync_chi=*/false, /*theta_gated=*/true);
    // joined whatever happened, so that nothing of this call runs on after it returns
    QR_CUDA_TRY(cudaEventRecord(bs->done[q], bs->st[q]));
    QR_CUDA_TRY(cudaStreamWaitEvent(st, bs->done[q], 0));
  }
  if (rc != QRTEBD_OK) return rc;
  // 3. one cut over all blocks
  QR_CUDA_TRY(cudaMemsetAsync(merged, 0, (size_t)p.eta_sum * sizeof(double), st));
  SymCutArgs ca{S, stq, merged, out_i, scal, io->stats_out, err, tr->chi_max, tr->svd_min,
                tr->tie_tol, tr->eps_target};
  k_sym_cut<<<1, 512, 0, st>>>(m, ca);
  note_launch();
  QR_CUDA_TRY(cudaGetLastError());
  // 4. scatter into the dense outputs
  {
    const long long n1 = p.nrows * cap;
    k_sym_scatter_bm<T><<<(unsigned)ceil_div(n1, 256), 256, 0, st>>>(
        bmq, rowsec, rowpos, out_i, m, static_cast<cx<T>*>(io->bm_out), p.nrows, cap);
    note_launch();
    const long long n2 = p.ncols * cap;
    k_sym_scatter_bn<T><<<(unsigned)ceil_div(n2, 256), 256, 0, st>>>(
        bnq, colsec, colpos, out_i, m, static_cast<cx<T>*>(io->bn_out), p.ncols, cap);
    note_launch();
    k_sym_xi<T><<<(unsigned)ceil_div(cap, 256), 256, 0, st>>>(S, out_i, m, scal,
                                                            static_cast<cx<T>*>(io->xi_out), cap);
    note_launch();
    QR_CUDA_TRY(cudaGetLastError());
  }
  int host_i[3 * kSymMaxD + 2];
  QR_CUDA_TRY(cudaMemcpyAsync(host_i, out_i, (2 * d + 1) * sizeof(int), cudaMemcpyDeviceToHost, st));
  QR_CUDA_TRY(cudaStreamSynchronize(st));
  const int chi_new = host_i[2 * d];
  if (chi_new < 1 || chi_new > cap) { set_last_message("sym_bond_update: bad cut"); return QRTEBD_ERR_NUMERIC; }
  int g = 0;
  for (int q = 0; q < d; ++q) {
    if (io->chi_sector_out) io->chi_sector_out[q] = host_i[q];
    for (int k = 0; k < host_i[q]; ++k) io->charge_out[g++] = q;
  }
  if (info) { info->eta = p.eta_sum; info->chi_new = chi_new; }
  return QRTEBD_OK;
}

}  // namespace

int sym_bond_update(const qrtebd_sym_bond_io* io, const qrtebd_trunc* tr, cudaStream_t st,
                    qrtebd_bond_info* info, size_t* bytes, int* eta_sum) {
  if (!io || !tr) return QRTEBD_ERR_INVALID_ARG;
  if (tr->sweeps < 0 || tr->sweeps > 1000) return QRTEBD_ERR_INVALID_ARG;
  switch (io->precision) {
    case QRTEBD_C128:
    case QRTEBD_C128_OZ: return sym_update_t<double>(io, tr, st, info, bytes, eta_sum);
    case QRTEBD_C64_3XTF32:
    case QRTEBD_C64_TF32:
    case QRTEBD_C64_FP32: return sym_update_t<float>(io, tr, st, info, bytes, eta_sum);
    default: return QRTEBD_ERR_INVALID_ARG;
  }
}

}  // namespace qrtebd

extern "C" {

int qrtebd_sym_bond_workspace_size(int precision, int chi_l, int d, int chi_m, int chi_r,
                                   const int* charge_l, const int* charge_m, const int* charge_r,
                                   int xi_kind, int theta_given, const qrtebd_trunc* tr,
                                   size_t* bytes, int* eta_sum) {
  if (!bytes || !tr) return QRTEBD_ERR_INVALID_ARG;
  qrtebd_sym_bond_io io;
  std::memset(&io, 0, sizeof io);
  static const char dummy = 0;
  io.bm = theta_given ? nullptr : &dummy;
  io.precision = precision;
  io.chi_l = chi_l; io.d = d; io.chi_m = chi_m; io.chi_r = chi_r;
  io.charge_l = charge_l; io.charge_m = charge_m; io.charge_r = charge_r;
  io.xi_kind = xi_kind;
  return qrtebd::sym_bond_update(&io, tr, nullptr, nullptr, bytes, eta_sum);
}

int qrtebd_sym_bond_update(const qrtebd_sym_bond_io* io, const qrtebd_trunc* tr, void* stream,
                           qrtebd_bond_info* info) {
  return qrtebd::sym_bond_update(io, tr, static_cast<cudaStream_t>(stream), info, nullptr, nullptr);
}

}  // extern "C"
