// Device-resident MPS and the TEBD layer driver (Sec. II, Fig. 1, Fig. 2a).
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "mps_impl.cuh"



namespace qrtebd {
namespace {

int site_count(const qrtebd_mps* s) { return s->L; }
int gate_count(const qrtebd_mps* s) { return s->infinite ? s->L : s->L - 1; }
int bond_index(const qrtebd_mps* s, int b) { return s->infinite ? ((b % s->L) + s->L) % s->L : b; }

template <typename T> __global__ void k_c128_to(const double2* in, cx<T>* out, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) out[i] = mk<T>((T)in[i].x, (T)in[i].y);
}
template <typename T> __global__ void k_to_c128v(const cx<T>* in, double2* out, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) out[i] = make_double2((double)in[i].x, (double)in[i].y);
}
// the diagonal of the dense n x n bond matrix, n = the cut chi~ read from stats[3] on the device
template <typename T> __global__ void k_diag_of(const cx<T>* M, const double* stats, int cap, cx<T>* v) {
  const int n = (int)stats[3];
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && i < cap) v[i] = M[(long long)i * n + i];
}
__global__ void k_acc_eps(const double* stats, double* acc, double* layer_slot) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    *acc += stats[0];
    if (layer_slot) *layer_slot = stats[0];
  }
}
// sum conj(x) y in FP64 (single pass, per-block partials then one block)
template <typename T>
__global__ void k_cdot_partial(const cx<T>* x, const cx<T>* y, long long n, double2* part) {
  double re = 0, im = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    cx<T> a = x[i], b = y[i];
    re += (double)a.x * b.x + (double)a.y * b.y;
    im += (double)a.x * b.y - (double)a.y * b.x;
  }
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
  }
  __shared__ double sr[32], si[32];
  if ((threadIdx.x & 31) == 0) { sr[threadIdx.x >> 5] = re; si[threadIdx.x >> 5] = im; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a += sr[w]; b += si[w]; }
    part[blockIdx.x] = make_double2(a, b);
  }
}
__global__ void k_sum2(const double2* part, int n, double2* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double a = 0, b = 0;
    for (int i = 0; i < n; ++i) { a += part[i].x; b += part[i].y; }
    *out = make_double2(a, b);
  }
}

long long sat_pow(int d, int e, long long cap) {
  long long v = 1;
  for (int i = 0; i < e; ++i) { v *= d; if (v >= cap) return cap; }
  return v;
}

int dev_alloc(void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 256;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) { (void)cudaGetLastError(); set_last_message("cudaMalloc failed"); return QRTEBD_ERR_OOM; }
  return QRTEBD_OK;
}

void free_all(qrtebd_mps* s) {
  for (void* p : s->B) cudaFree(p);
  for (void* p : s->Xi) cudaFree(p);
  for (void* p : s->xiv) cudaFree(p);
  cudaFree(s->eps_acc); cudaFree(s->stats); cudaFree(s->layer_eps); cudaFree(s->gates);
  cudaFree(s->ws); cudaFree(s->aux);
  s->B.clear(); s->Xi.clear(); s->xiv.clear();
}

int ensure_ws(qrtebd_mps* s, size_t need) {
  if (need <= s->ws_bytes) return QRTEBD_OK;
  QR_CUDA_TRY(cudaStreamSynchronize(s->st));
  cudaFree(s->ws);
  s->ws = nullptr; s->ws_bytes = 0;
  QR_TRY(dev_alloc(&s->ws, need));
  s->ws_bytes = need;
  return QRTEBD_OK;
}
int ensure_aux(qrtebd_mps* s, size_t need) {
  if (need <= s->aux_bytes) return QRTEBD_OK;
  QR_CUDA_TRY(cudaStreamSynchronize(s->st));
  cudaFree(s->aux);
  s->aux = nullptr; s->aux_bytes = 0;
  QR_TRY(dev_alloc(&s->aux, need));
  s->aux_bytes = need;
  return QRTEBD_OK;
}

int allocate(qrtebd_mps* s) {
  const int L = s->L, d = s->d;
  s->nbonds_store = s->infinite ? L : L + 1;
  s->chi.assign(s->nbonds_store, 1);
  s->cap.resize(s->nbonds_store);
  for (int b = 0; b < s->nbonds_store; ++b)
    s->cap[b] = s->infinite ? s->chi_max
                            : (int)std::min<long long>(std::min(sat_pow(d, b, s->chi_max),
                                                                sat_pow(d, L - b, s->chi_max)),
                                                       s->chi_max);
  if (!s->infinite) { s->cap[0] = 1; s->cap[L] = 1; }
  s->B.assign(L, nullptr);
  s->Xi.assign(s->nbonds_store, nullptr);
  s->xiv.assign(s->nbonds_store, nullptr);
  s->xi_diag.assign(s->nbonds_store, 1);
  s->xi_lower.assign(s->nbonds_store, 0);
  s->chi_pending.assign(s->nbonds_store, 0);
  for (int m = 0; m < L; ++m) {
    int r = s->infinite ? (m + 1) % L : m + 1;
    QR_TRY(dev_alloc(&s->B[m], (size_t)s->cap[m] * d * s->cap[r] * s->esz));
  }
  for (int b = 0; b < s->nbonds_store; ++b) {
    QR_TRY(dev_alloc(&s->Xi[b], (size_t)s->cap[b] * s->cap[b] * s->esz));
    QR_TRY(dev_alloc(&s->xiv[b], (size_t)s->cap[b] * s->esz));
  }
  QR_TRY(dev_alloc((void**)&s->eps_acc, s->nbonds_store * sizeof(double)));
  QR_TRY(dev_alloc((void**)&s->stats, 4 * (size_t)(gate_count(s) + 1) * sizeof(double)));
  QR_TRY(dev_alloc((void**)&s->layer_eps, (gate_count(s) + 1) * sizeof(double)));
  QR_TRY(dev_alloc((void**)&s->gates, (size_t)(gate_count(s) + 1) * d * d * d * d * sizeof(double2)));
  QR_CUDA_TRY(cudaMemsetAsync(s->eps_acc, 0, s->nbonds_store * sizeof(double), s->st));
  // the bond-update workspace is allocated on first use (single-state layers);
  // batched layers use the executor's per-worker workspaces instead
  return QRTEBD_OK;
}

template <typename T> int init_product(qrtebd_mps* s, const double* amps) {
  const int L = s->L, d = s->d;
  std::vector<cx<T>> h((size_t)d);
  for (int m = 0; m < L; ++m) {
    for (int i = 0; i < d; ++i)
      h[i] = amps ? mk<T>((T)amps[2 * (m * d + i)], (T)amps[2 * (m * d + i) + 1])
                  : mk<T>(i == 0 ? T(1) : T(0), T(0));
    QR_CUDA_TRY(cudaMemcpyAsync(s->B[m], h.data(), d * sizeof(cx<T>), cudaMemcpyHostToDevice, s->st));
    QR_CUDA_TRY(cudaStreamSynchronize(s->st));
  }
  cx<T> one = mk<T>(1, 0);
  for (int b = 0; b < s->nbonds_store; ++b) {
    QR_CUDA_TRY(cudaMemcpyAsync(s->Xi[b], &one, sizeof one, cudaMemcpyHostToDevice, s->st));
    QR_CUDA_TRY(cudaMemcpyAsync(s->xiv[b], &one, sizeof one, cudaMemcpyHostToDevice, s->st));
    QR_CUDA_TRY(cudaStreamSynchronize(s->st));
  }
  return QRTEBD_OK;
}

template <typename T>
int update_bond_t(qrtebd_mps* s, int m, const qrtebd_trunc* tr, cudaStream_t st, void* ws,
                  size_t ws_bytes) {
  const int d = s->d, d4 = d * d * d * d;
  const int n = s->infinite ? (m + 1) % s->L : m + 1;
  const int bl = bond_index(s, m), bmid = bond_index(s, m + 1), br = bond_index(s, m + 2);
  qrtebd_bond_io io;
  std::memset(&io, 0, sizeof io);
  io.precision = s->precision;
  io.chi_l = s->chi[bl]; io.d = d; io.chi_m = s->chi[bmid]; io.chi_r = s->chi[br];
  const bool diag = s->xi_diag[bl] != 0;
  io.xi_kind = diag ? 2 : (s->xi_lower[bl] ? 3 : 1);
  io.xi = diag ? s->xiv[bl] : s->Xi[bl];
  io.bm = s->B[m]; io.bn = s->B[n];
  io.gate = s->gates + (size_t)m * d4;
  io.bm_out = s->B[m]; io.bn_out = s->B[n]; io.xi_out = s->Xi[bmid];
  io.stats_out = s->stats + 4 * (size_t)m;
  io.workspace = ws; io.workspace_bytes = ws_bytes;
  qrtebd_trunc t = *tr;
  if (t.chi_max > s->cap[bmid]) t.chi_max = s->cap[bmid];
  qrtebd_bond_info info;
  // no host synchronisation: a CBE cut stays on the device (stats[3]) until mps_collect_cuts
  QR_TRY(bond_update(&io, &t, st, &info, nullptr, /*sync_chi=*/false));
  if (t.scheme == QRTEBD_CBE) {
    s->chi_pending[bmid] = 1;
    s->xi_lower[bmid] = 0;
    k_diag_of<T><<<(unsigned)ceil_div(s->cap[bmid], 128), 128, 0, st>>>(
        static_cast<cx<T>*>(s->Xi[bmid]), s->stats + 4 * (size_t)m, s->cap[bmid],
        static_cast<cx<T>*>(s->xiv[bmid]));
    note_launch();
  } else {
    s->chi[bmid] = info.chi_new;
    s->xi_diag[bmid] = 0;
    s->xi_lower[bmid] = 1;  // Xi~ = L / ||L||
  }
  k_acc_eps<<<1, 1, 0, st>>>(s->stats + 4 * (size_t)m, s->eps_acc + bmid, s->layer_eps + m);
  note_launch();
  QR_CUDA_TRY(cudaGetLastError());
  return QRTEBD_OK;
}

template <typename T>
int apply_layer_t(qrtebd_mps* s, int parity, const double* gates_host, const qrtebd_trunc* tr,
                  double* eps_out) {
  const int ng = gate_count(s);
  QR_TRY(mps_upload_gates(s, parity, gates_host));
  for (int m = parity; m < ng; m += 2) {
    size_t need = 0;
    QR_TRY(mps_bond_ws_need(s, m, tr, &need));
    QR_TRY(ensure_ws(s, need));
    QR_TRY(update_bond_t<T>(s, m, tr, s->st, s->ws, s->ws_bytes));
  }
  QR_TRY(mps_collect_cuts(s));
  if (eps_out) {
    std::vector<double> le(ng + 1);
    QR_CUDA_TRY(cudaMemcpyAsync(le.data(), s->layer_eps, ng * sizeof(double), cudaMemcpyDeviceToHost, s->st));
    QR_CUDA_TRY(cudaStreamSynchronize(s->st));
    for (int m = parity; m < ng; m += 2) eps_out[m] = le[m];
  }
  return QRTEBD_OK;
}

template <typename T> int cdot(const cx<T>* x, const cx<T>* y, long long n, double2* part,
                               double2* out, cudaStream_t st) {
  k_cdot_partial<T><<<148, 256, 0, st>>>(x, y, n, part);
  note_launch();
  k_sum2<<<1, 1, 0, st>>>(part, 148, out);
  note_launch();
  QR_CUDA_TRY(cudaGetLastError());
  return QRTEBD_OK;
}

template <typename T>
int expectation_t(qrtebd_mps* s, int site, int nsites, const double* op_host, double* out) {
  const int d = s->d, L = s->L;
  if (site < 0 || site >= L || (nsites != 1 && nsites != 2)) return QRTEBD_ERR_INVALID_ARG;
  if (nsites == 2 && !s->infinite && site + 1 >= L) return QRTEBD_ERR_INVALID_ARG;
  const int n = s->infinite ? (site + 1) % L : site + 1;
  const int bl = bond_index(s, site), bmid = bond_index(s, site + 1), br = bond_index(s, site + 2);
  const long long chiL = s->chi[bl], chiM = s->chi[bmid], chiR = s->chi[br];
  const int k = nsites == 1 ? d : d * d;
  const long long rest = nsites == 1 ? d * chiM : d * d * chiR;
  const long long nel = chiL * rest;
  size_t need = (size_t)(3 * nel + 2 * nsites * nsites * d * d + (size_t)k * k + 300) * sizeof(cx<T>) +
                (size_t)k * k * sizeof(double2) + 2048;
  if (nsites == 2) need += (size_t)chiL * d * chiM * sizeof(cx<T>);
  QR_TRY(ensure_aux(s, need));
  Arena ar; ar.base = static_cast<char*>(s->aux); ar.cap = s->aux_bytes;
  cx<T>* C = ar.take<cx<T>>(nel);
  cx<T>* D = ar.take<cx<T>>(nel);
  cx<T>* XB = nsites == 2 ? ar.take<cx<T>>(chiL * d * chiM) : nullptr;
  double2* O64 = ar.take<double2>((size_t)k * k);
  cx<T>* Ot = ar.take<cx<T>>((size_t)k * k);
  double2* part = ar.take<double2>(160);
  double2* res = ar.take<double2>(2);
  if (ar.overflow()) return QRTEBD_ERR_OOM;
  QR_CUDA_TRY(cudaMemcpyAsync(O64, op_host, (size_t)k * k * sizeof(double2), cudaMemcpyHostToDevice, s->st));
  k_c128_to<T><<<(unsigned)ceil_div((long long)k * k, 128), 128, 0, s->st>>>(O64, Ot, (long long)k * k);
  note_launch();
  const cx<T> one = mk<T>(1, 0), zero = mk<T>(0, 0);
  const bool diag = s->xi_diag[bl] != 0;
  // C = Xi B^m (and then B^n for two sites)
  const cx<T>* Bm = static_cast<const cx<T>*>(s->B[site]);
  cx<T>* XBm = nsites == 1 ? C : XB;
  {
    GemmArgs<T> g{(int)chiL, (int)(d * chiM), (int)chiL, static_cast<const cx<T>*>(s->Xi[bl]), chiL, 1,
                  false, Bm, d * chiM, 1, false, XBm, d * chiM, 1, one, zero};
    (void)diag;  // the dense copy of Xi is always valid
    QR_TRY(gemm_simt<T>(g, s->st));
  }
  if (nsites == 2) {
    GemmArgs<T> g{(int)(chiL * d), (int)(d * chiR), (int)chiM, XB, chiM, 1, false,
                  static_cast<const cx<T>*>(s->B[n]), d * chiR, 1, false, C, d * chiR, 1, one, zero};
    QR_TRY(gemm_simt<T>(g, s->st));
  }
  // D[a] = O C[a] for every left index a: batched (k x k) . (k x cols)
  const long long cols = nsites == 1 ? chiM : chiR;
  {
    GemmArgs<T> g{k, (int)cols, k, Ot, k, 1, false, C, cols, 1, false, D, cols, 1, one, zero};
    g.batch = (int)chiL; g.bsa = 0; g.bsb = (long long)k * cols; g.bsc = g.bsb;
    QR_TRY(gemm_simt<T>(g, s->st));
  }
  QR_TRY(cdot<T>(C, D, nel, part, res, s->st));
  double2 h;
  QR_CUDA_TRY(cudaMemcpyAsync(&h, res, sizeof h, cudaMemcpyDeviceToHost, s->st));
  QR_CUDA_TRY(cudaStreamSynchronize(s->st));
  out[0] = h.x; out[1] = h.y;
  return QRTEBD_OK;
}

template <typename T> int schmidt_t(qrtebd_mps* s, int b, double* S, int capacity, int* n) {
  const int c = s->chi[b];
  *n = c;
  if (capacity < c) return QRTEBD_ERR_INVALID_ARG;
  std::vector<double> sv(c);
  if (s->xi_diag[b]) {
    std::vector<cx<T>> h(c);
    QR_CUDA_TRY(cudaMemcpyAsync(h.data(), s->xiv[b], c * sizeof(cx<T>), cudaMemcpyDeviceToHost, s->st));
    QR_CUDA_TRY(cudaStreamSynchronize(s->st));
    for (int i = 0; i < c; ++i) sv[i] = std::sqrt((double)h[i].x * h[i].x + (double)h[i].y * h[i].y);
  } else if (svd64_supported(c)) {
    // the singular values of a dense Xi: one-sided FP64 Jacobi on its rows (Xi Xi^dag is never
    // formed; one cooperative launch)
    const long long cc = (long long)c * c;
    const size_t wb = svd64_work_bytes(c);
    size_t need = (size_t)(2 * cc + 64) * sizeof(double2) + c * sizeof(double) + wb + 4096;
    QR_TRY(ensure_aux(s, need));
    Arena ar; ar.base = static_cast<char*>(s->aux); ar.cap = s->aux_bytes;
    double2* X = ar.take<double2>(cc);
    double2* Vh = ar.take<double2>(cc);
    double* w = ar.take<double>(c);
    char* work = ar.take<char>(wb);
    if (ar.overflow()) return QRTEBD_ERR_OOM;
    k_to_c128v<T><<<(unsigned)ceil_div(cc, 256), 256, 0, s->st>>>(static_cast<const cx<T>*>(s->Xi[b]), X, cc);
    note_launch();
    QR_TRY(svd_rows_jacobi64(X, c, c, w, Vh, work, wb, s->st, device_error_word()));
    QR_CUDA_TRY(cudaMemcpyAsync(sv.data(), w, c * sizeof(double), cudaMemcpyDeviceToHost, s->st));
    QR_CUDA_TRY(cudaStreamSynchronize(s->st));
    for (double& x : sv) x = x > 0 ? std::sqrt(x) : 0.0;
  } else {
    const long long cc = (long long)c * c;
    size_t need = (size_t)(3 * cc + herm_eig_scratch_elems(c) + 64) * sizeof(double2) + c * sizeof(double) + 4096;
    QR_TRY(ensure_aux(s, need));
    Arena ar; ar.base = static_cast<char*>(s->aux); ar.cap = s->aux_bytes;
    double2* X = ar.take<double2>(cc);
    double2* M = ar.take<double2>(cc);
    double2* Vh = ar.take<double2>(cc);
    double* w = ar.take<double>(c);
    size_t se = herm_eig_scratch_elems(c);
    double2* scr = ar.take<double2>(se);
    if (ar.overflow()) return QRTEBD_ERR_OOM;
    k_to_c128v<T><<<(unsigned)ceil_div(cc, 256), 256, 0, s->st>>>(static_cast<const cx<T>*>(s->Xi[b]), X, cc);
    note_launch();
    GemmArgs<double> g{c, c, c, X, 1, c, true, X, c, 1, false, M, c, 1, mk<double>(1, 0), mk<double>(0, 0)};
    QR_TRY(gemm_simt<double>(g, s->st));
    QR_TRY(herm_eig(M, c, w, Vh, scr, se, s->st, device_error_word()));
    QR_CUDA_TRY(cudaMemcpyAsync(sv.data(), w, c * sizeof(double), cudaMemcpyDeviceToHost, s->st));
    QR_CUDA_TRY(cudaStreamSynchronize(s->st));
    for (double& x : sv) x = x > 0 ? std::sqrt(x) : 0.0;
  }
  std::sort(sv.begin(), sv.end(), [](double a, double b2) { return a > b2; });
  double nrm = 0;
  for (double x : sv) nrm += x * x;
  nrm = std::sqrt(nrm);
  for (int i = 0; i < c; ++i) S[i] = nrm > 0 ? sv[i] / nrm : 0.0;
  return QRTEBD_OK;
}

const unsigned kMagic = 0x51525442u;  // "QRTB"

}  // namespace

int mps_gate_count(const qrtebd_mps* s) { return gate_count(s); }

int mps_upload_gates(qrtebd_mps* s, int parity, const double* gates_host) {
  const int d = s->d, d4 = d * d * d * d, ng = gate_count(s);
  for (int m = parity; m < ng; m += 2)
    QR_CUDA_TRY(cudaMemcpyAsync(s->gates + (size_t)m * d4, gates_host + 2 * (size_t)m * d4,
                                d4 * sizeof(double2), cudaMemcpyHostToDevice, s->st));
  return QRTEBD_OK;
}

int mps_bond_ws_need(const qrtebd_mps* s, int m, const qrtebd_trunc* tr, size_t* need) {
  const int bl = bond_index(s, m), bmid = bond_index(s, m + 1), br = bond_index(s, m + 2);
  qrtebd_bond_io io;
  std::memset(&io, 0, sizeof io);
  io.precision = s->precision;
  io.chi_l = s->chi[bl]; io.d = s->d; io.chi_m = s->chi[bmid]; io.chi_r = s->chi[br];
  io.xi_kind = s->xi_diag[bl] ? 2 : (s->xi_lower[bl] ? 3 : 1);
  static const char dummy = 0;
  io.bm = &dummy;
  qrtebd_trunc t = *tr;
  if (t.chi_max > s->cap[bmid]) t.chi_max = s->cap[bmid];
  return bond_update(&io, &t, nullptr, nullptr, need);
}

int mps_collect_cuts(qrtebd_mps* s) {
  bool any = false;
  for (char c : s->chi_pending) any = any || c;
  if (!any) return QRTEBD_OK;
  const int ng = gate_count(s);
  std::vector<double> st(4 * (size_t)ng);
  QR_CUDA_TRY(cudaMemcpyAsync(st.data(), s->stats, st.size() * sizeof(double), cudaMemcpyDeviceToHost, s->st));
  QR_CUDA_TRY(cudaStreamSynchronize(s->st));
  for (int m = 0; m < ng; ++m) {
    const int bmid = bond_index(s, m + 1);
    if (!s->chi_pending[bmid]) continue;
    const int c = (int)st[4 * (size_t)m + 3];
    if (c < 1 || c > s->cap[bmid]) { set_last_message("CBE: bad cut"); return QRTEBD_ERR_NUMERIC; }
    s->chi[bmid] = c;
    s->xi_diag[bmid] = 1;
    s->chi_pending[bmid] = 0;
  }
  return QRTEBD_OK;
}

int mps_update_bond(qrtebd_mps* s, int m, const qrtebd_trunc* tr, cudaStream_t st, void* ws,
                    size_t ws_bytes) {
  return prec_is_c128(s->precision) ? update_bond_t<double>(s, m, tr, st, ws, ws_bytes)
                                     : update_bond_t<float>(s, m, tr, st, ws, ws_bytes);
}

}  // namespace qrtebd

using namespace qrtebd;

extern "C" {

int qrtebd_mps_create(const qrtebd_mps_desc* desc, void* stream, qrtebd_mps** out) {
  if (!desc || !out) return QRTEBD_ERR_INVALID_ARG;
  *out = nullptr;
  if (desc->d < 2 || desc->d > 8 || desc->chi_max < 1 || desc->L < 2) return QRTEBD_ERR_INVALID_ARG;
  if (desc->infinite && (desc->L % 2)) return QRTEBD_ERR_INVALID_ARG;
  if (!prec_valid(desc->precision)) return QRTEBD_ERR_INVALID_ARG;
  qrtebd_mps* s = new qrtebd_mps();
  s->L = desc->L; s->d = desc->d; s->infinite = desc->infinite ? 1 : 0;
  s->chi_max = desc->chi_max; s->precision = desc->precision;
  s->st = static_cast<cudaStream_t>(stream);
  s->esz = prec_is_c128(desc->precision) ? sizeof(double2) : sizeof(float2);
  int rc = allocate(s);
  if (rc == QRTEBD_OK)
    rc = prec_is_c128(desc->precision) ? init_product<double>(s, desc->product_state)
                                        : init_product<float>(s, desc->product_state);
  if (rc != QRTEBD_OK) { free_all(s); delete s; return rc; }
  *out = s;
  return QRTEBD_OK;
}

int qrtebd_mps_destroy(qrtebd_mps* s) {
  if (!s) return QRTEBD_OK;
  executor_forget_state(s);
  cudaDeviceSynchronize();  // batched layers may still run on the executor's streams
  free_all(s);
  delete s;
  return QRTEBD_OK;
}

int qrtebd_apply_gate_layer(qrtebd_mps* s, int parity, const double* gates_host,
                            const qrtebd_trunc* tr, double* eps_out) {
  if (!s || !gates_host || !tr || (parity != 0 && parity != 1)) return QRTEBD_ERR_INVALID_ARG;
  // The bonds of one parity are independent (Fig. 2a): with two or more of them the layer
  // runs on the executor's worker streams, side by side (and, plain scheme, as a replayed
  // CUDA graph once its shapes repeat); a single bond runs on the state's own stream.
  if ((gate_count(s) - parity + 1) / 2 >= 2) {
    qrtebd_mps* const states[1] = {s};
    const double* const gates[1] = {gates_host};
    double* const eps[1] = {eps_out};
    return qrtebd_apply_gate_layer_batched(states, 1, parity, gates, tr, eps);
  }
  return prec_is_c128(s->precision) ? apply_layer_t<double>(s, parity, gates_host, tr, eps_out)
                                     : apply_layer_t<float>(s, parity, gates_host, tr, eps_out);
}

int qrtebd_expectation(qrtebd_mps* s, int site, int nsites, const double* op_host, double* out) {
  if (!s || !op_host || !out) return QRTEBD_ERR_INVALID_ARG;
  return prec_is_c128(s->precision) ? expectation_t<double>(s, site, nsites, op_host, out)
                                     : expectation_t<float>(s, site, nsites, op_host, out);
}

int qrtebd_truncation_error(qrtebd_mps* s, int bond, double* out) {
  if (!s || !out) return QRTEBD_ERR_INVALID_ARG;
  std::vector<double> h(s->nbonds_store);
  QR_CUDA_TRY(cudaMemcpyAsync(h.data(), s->eps_acc, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s->st));
  QR_CUDA_TRY(cudaStreamSynchronize(s->st));
  if (bond == -1) {
    double t = 0;
    for (double x : h) t += x;
    *out = t;
    return QRTEBD_OK;
  }
  if (bond < 0 || (!s->infinite && bond > s->L)) return QRTEBD_ERR_INVALID_ARG;
  *out = h[bond_index(s, bond)];
  return QRTEBD_OK;
}

int qrtebd_schmidt(qrtebd_mps* s, int bond, double* S, int capacity, int* n) {
  if (!s || !S || !n || bond < 0 || bond >= (s->infinite ? s->L : s->L + 1)) return QRTEBD_ERR_INVALID_ARG;
  return prec_is_c128(s->precision) ? schmidt_t<double>(s, bond, S, capacity, n)
                                     : schmidt_t<float>(s, bond, S, capacity, n);
}

int qrtebd_entropy(qrtebd_mps* s, int bond, double* out) {
  if (!s || !out || bond < 0 || bond >= (s->infinite ? s->L : s->L + 1)) return QRTEBD_ERR_INVALID_ARG;
  std::vector<double> S((size_t)std::max(s->chi[bond], 1));
  int n = 0;
  QR_TRY(qrtebd_schmidt(s, bond, S.data(), (int)S.size(), &n));
  // S is normalised to unit 2-norm, so p_k = S_k^2 sums to one; FP64, natural log
  double e = 0.0;
  for (int k = 0; k < n; ++k) {
    const double p = S[k] * S[k];
    if (p > 1e-300) e -= p * std::log(p);
  }
  *out = e;
  return QRTEBD_OK;
}

int qrtebd_bond_dims(qrtebd_mps* s, int* dims, int capacity, int* n) {
  if (!s || !dims || !n) return QRTEBD_ERR_INVALID_ARG;
  *n = s->nbonds_store;
  if (capacity < s->nbonds_store) return QRTEBD_ERR_INVALID_ARG;
  for (int b = 0; b < s->nbonds_store; ++b) dims[b] = s->chi[b];
  return QRTEBD_OK;
}

int qrtebd_sync(qrtebd_mps* s) {
  if (!s) return QRTEBD_ERR_INVALID_ARG;
  return qrtebd_stream_check(s->st);
}

int qrtebd_mps_save(qrtebd_mps* s, const char* path) {
  if (!s || !path) return QRTEBD_ERR_INVALID_ARG;
  QR_CUDA_TRY(cudaStreamSynchronize(s->st));
  FILE* f = fopen(path, "wb");
  if (!f) { set_last_message("mps_save: cannot open file"); return QRTEBD_ERR_INVALID_ARG; }
  int hdr[6] = {(int)kMagic, s->L, s->d, s->infinite, s->chi_max, s->precision};
  bool ok = fwrite(hdr, sizeof hdr, 1, f) == 1;
  ok = ok && fwrite(s->chi.data(), sizeof(int), s->chi.size(), f) == s->chi.size();
  ok = ok && fwrite(s->xi_diag.data(), 1, s->xi_diag.size(), f) == s->xi_diag.size();
  std::vector<char> buf;
  auto dump = [&](const void* dptr, size_t bytes) {
    buf.resize(bytes);
    if (bytes && cudaMemcpy(buf.data(), dptr, bytes, cudaMemcpyDeviceToHost) != cudaSuccess) return false;
    return fwrite(buf.data(), 1, bytes, f) == bytes;
  };
  for (int m = 0; ok && m < s->L; ++m) {
    int r = s->infinite ? (m + 1) % s->L : m + 1;
    ok = dump(s->B[m], (size_t)s->chi[m] * s->d * s->chi[r] * s->esz);
  }
  for (int b = 0; ok && b < s->nbonds_store; ++b) {
    ok = dump(s->Xi[b], (size_t)s->chi[b] * s->chi[b] * s->esz);
    ok = ok && dump(s->xiv[b], (size_t)s->chi[b] * s->esz);
  }
  ok = ok && dump(s->eps_acc, s->nbonds_store * sizeof(double));
  fclose(f);
  if (!ok) { set_last_message("mps_save: write failed"); return QRTEBD_ERR_CUDA; }
  return QRTEBD_OK;
}

int qrtebd_mps_load(const char* path, void* stream, qrtebd_mps** out) {
  if (!path || !out) return QRTEBD_ERR_INVALID_ARG;
  *out = nullptr;
  FILE* f = fopen(path, "rb");
  if (!f) { set_last_message("mps_load: cannot open file"); return QRTEBD_ERR_INVALID_ARG; }
  auto reject = [&](const char* why) { fclose(f); set_last_message(why); return QRTEBD_ERR_INVALID_ARG; };
  int hdr[6];
  if (fread(hdr, sizeof hdr, 1, f) != 1 || hdr[0] != (int)kMagic) return reject("mps_load: not a qrtebd checkpoint");
  const int L = hdr[1], d = hdr[2], inf = hdr[3], chi_max = hdr[4], prec = hdr[5];
  if (d < 2 || d > 8 || chi_max < 1 || L < 2 || L > (1 << 20) || (inf != 0 && inf != 1) || (inf && L % 2) ||
      !prec_valid(prec))
    return reject("mps_load: corrupt header");
  // Everything is checked on the host before any device memory is taken: the bond
  // dimensions against the capacities mps_create gives, and the file length against
  // the bytes those dimensions imply, so that a truncated or padded file is refused.
  const int nb = inf ? L : L + 1;
  std::vector<int> chi(nb);
  std::vector<char> diag(nb);
  if (fread(chi.data(), sizeof(int), nb, f) != (size_t)nb || fread(diag.data(), 1, nb, f) != (size_t)nb)
    return reject("mps_load: truncated or corrupt file");
  const size_t esz = prec_is_c128(prec) ? sizeof(double2) : sizeof(float2);
  size_t body = (size_t)nb * sizeof(double);
  for (int b = 0; b < nb; ++b) {
    const long long cap = inf ? chi_max
                              : (b == 0 || b == L) ? 1
                              : std::min<long long>(std::min(sat_pow(d, b, chi_max), sat_pow(d, L - b, chi_max)),
                                                    chi_max);
    if (chi[b] < 1 || chi[b] > cap) return reject("mps_load: bond dimension out of range");
    body += ((size_t)chi[b] * chi[b] + chi[b]) * esz;
  }
  for (int m = 0; m < L; ++m) body += (size_t)chi[m] * d * chi[inf ? (m + 1) % L : m + 1] * esz;
  const long long here = ftell(f);
  if (here < 0 || fseek(f, 0, SEEK_END) != 0) return reject("mps_load: cannot read file");
  const long long total = ftell(f);
  if (total != here + (long long)body || fseek(f, here, SEEK_SET) != 0)
    return reject("mps_load: truncated or corrupt file");
  qrtebd_mps_desc desc{L, d, inf, chi_max, prec, nullptr};
  qrtebd_mps* s = nullptr;
  int rc = qrtebd_mps_create(&desc, stream, &s);
  if (rc != QRTEBD_OK) { fclose(f); return rc; }
  s->chi = chi;
  for (int b = 0; b < nb; ++b) s->xi_diag[b] = diag[b];
  bool ok = true;
  std::vector<char> buf;
  auto load = [&](void* dptr, size_t bytes) {
    buf.resize(bytes);
    if (fread(buf.data(), 1, bytes, f) != bytes) return false;
    return !bytes || cudaMemcpy(dptr, buf.data(), bytes, cudaMemcpyHostToDevice) == cudaSuccess;
  };
  for (int m = 0; ok && m < s->L; ++m) {
    int r = s->infinite ? (m + 1) % s->L : m + 1;
    ok = load(s->B[m], (size_t)s->chi[m] * s->d * s->chi[r] * s->esz);
  }
  for (int b = 0; ok && b < s->nbonds_store; ++b) {
    ok = load(s->Xi[b], (size_t)s->chi[b] * s->chi[b] * s->esz);
    ok = ok && load(s->xiv[b], (size_t)s->chi[b] * s->esz);
  }
  ok = ok && load(s->eps_acc, s->nbonds_store * sizeof(double));
  fclose(f);
  if (!ok) { qrtebd_mps_destroy(s); set_last_message("mps_load: truncated or corrupt file"); return QRTEBD_ERR_INVALID_ARG; }
  *out = s;
  return QRTEBD_OK;
}

}  // extern "C"
