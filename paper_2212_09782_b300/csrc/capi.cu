// extern "C" entry points of libqrtebd (declared in include/qrtebd.h).
#include <complex>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "bond.cuh"
#include "tc_gemm.cuh"

namespace qrtebd {

namespace {
__device__ unsigned g_dev_err;  // device error word (one per device)
thread_local std::string g_msg;
std::mutex g_err_mu;
unsigned* g_err_ptr[64] = {};
}  // namespace

void set_last_error(cudaError_t e, const char* what, const char* file, int line) {
  char buf[512];
  snprintf(buf, sizeof buf, "%s: %s (%s:%d)", cudaGetErrorString(e), what, file, line);
  g_msg = buf;
}
void set_last_message(const char* msg) { g_msg = msg; }

unsigned* device_error_word() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(g_err_mu);
  if (!g_err_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_dev_err) != cudaSuccess) return nullptr;
    g_err_ptr[dev] = static_cast<unsigned*>(p);
  }
  return g_err_ptr[dev];
}

std::vector<const void*>& barrier_spin_symbols() {
  static std::vector<const void*> v;
  return v;
}
std::mutex& barrier_spin_mu() {
  static std::mutex m;
  return m;
}
int register_barrier_spin(const void* host_symbol) {
  std::lock_guard<std::mutex> lk(barrier_spin_mu());
  barrier_spin_symbols().push_back(host_symbol);
  return (int)barrier_spin_symbols().size();
}

namespace {
__device__ unsigned g_selftest_bar[2];
// One CTA waits at a grid barrier sized for two: the counter that would release it is never
// advanced, so the bounded wait runs out, sets DEVERR_TIMEOUT and the kernel returns.
__global__ void k_selftest_barrier(unsigned* bar, unsigned* err) { (void)grid_barrier(bar, 2u, err); }
}  // namespace

// Read-and-clear the device error word (synchronises the stream first).
int check_device_error(cudaStream_t st) {
  QR_CUDA_TRY(cudaStreamSynchronize(st));
  unsigned* p = device_error_word();
  if (!p) { set_last_message("device error word unavailable"); return QRTEBD_ERR_CUDA; }
  unsigned h = 0;
  QR_CUDA_TRY(cudaMemcpy(&h, p, sizeof h, cudaMemcpyDeviceToHost));
  if (h) {
    unsigned z = 0;
    QR_CUDA_TRY(cudaMemcpy(p, &z, sizeof z, cudaMemcpyHostToDevice));
    if (h & DEVERR_TIMEOUT) { set_last_message("a kernel gave up a bounded wait"); return QRTEBD_ERR_TIMEOUT; }
    if (h & DEVERR_NUMERIC) { set_last_message("NaN/Inf met in a norm"); return QRTEBD_ERR_NUMERIC; }
    set_last_message("device bounds check failed");
    return QRTEBD_ERR_INVALID_ARG;
  }
  return QRTEBD_OK;
}

// ---------------------------------------------------------------- clock gate
namespace {
using zc = std::complex<double>;

// Cyclic Jacobi for a small Hermitian matrix (host): A = V diag(w) V^dag.
void herm_jacobi_host(int n, std::vector<zc>& A, std::vector<zc>& V, std::vector<double>& w) {
  V.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0, tot = 0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        double a2 = std::norm(A[(size_t)i * n + j]);
        tot += a2;
        if (i != j) off += a2;
      }
    if (off <= 1e-32 * tot || tot == 0) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        zc apq = A[(size_t)p * n + q];
        double ab = std::abs(apq);
        if (ab < 1e-300) continue;
        double app = A[(size_t)p * n + p].real(), aqq = A[(size_t)q * n + q].real();
        double z = (aqq - app) / (2 * ab);
        double t = (z >= 0 ? 1.0 : -1.0) / (std::fabs(z) + std::sqrt(1 + z * z));
        double c = 1 / std::sqrt(1 + t * t), s = t * c;
        zc se = s * apq / ab;
        for (int i = 0; i < n; ++i) {  // columns: A G, V G
          zc x = A[(size_t)i * n + p], y = A[(size_t)i * n + q];
          A[(size_t)i * n + p] = c * x - std::conj(se) * y;
          A[(size_t)i * n + q] = se * x + c * y;
          x = V[(size_t)i * n + p]; y = V[(size_t)i * n + q];
          V[(size_t)i * n + p] = c * x - std::conj(se) * y;
          V[(size_t)i * n + q] = se * x + c * y;
        }
        for (int j = 0; j < n; ++j) {  // rows: G^dag A
          zc x = A[(size_t)p * n + j], y = A[(size_t)q * n + j];
          A[(size_t)p * n + j] = c * x - se * y;
          A[(size_t)q * n + j] = std::conj(se) * x + c * y;
        }
      }
  }
  w.resize(n);
  for (int i = 0; i < n; ++i) w[i] = A[(size_t)i * n + i].real();
}
}  // namespace

}  // namespace qrtebd

using namespace qrtebd;

namespace qrtebd {
namespace {
template <typename T>
int qr_entry(int precision, int m, int n, void* A, long long lda, void* Q, long long ldq,
             void* ws, size_t bytes, cudaStream_t st, size_t* need) {
  Arena ar;
  ar.measuring = (need != nullptr);
  if (!need) { ar.base = static_cast<char*>(ws); ar.cap = bytes; }
  QrScratch<T> qs;
  qr_carve<T>(ar, m, n, qs);
  TcWorkspace tcw, tcw_side;
  OzWorkspace ozw, ozw_side;
  const bool tc = std::is_same<T, float>::value &&
                  (precision == QRTEBD_C64_3XTF32 || precision == QRTEBD_C64_TF32);
  const bool oz = std::is_same<T, double>::value && precision == QRTEBD_C128_OZ;
  if (tc) tc_carve(ar, std::max(m, n), m, std::max(m, n), tcw);
  if (tc) tc_carve(ar, std::max(m, n), m, std::max(m, n), tcw_side);
  if (oz) oz_carve(ar, std::max(m, n), m, n, ozw);
  if (oz) oz_carve(ar, std::max(m, n), m, n, ozw_side);
  if (need) { *need = ar.off; return QRTEBD_OK; }
  if (ar.overflow() || !ws) { set_last_message("qr: workspace too small"); return QRTEBD_ERR_OOM; }
  struct Ctx { TcWorkspace* w; OzWorkspace* o; bool three; bool tc; bool oz; };
  Ctx ctx{&tcw, &ozw, precision == QRTEBD_C64_3XTF32, tc, oz};
  Ctx ctx_side{&tcw_side, &ozw_side, precision == QRTEBD_C64_3XTF32, tc, oz};
  auto fn = [](const GemmArgs<T>& g, cudaStream_t s, void* c) -> int {
    Ctx* x = static_cast<Ctx*>(c);
    if constexpr (std::is_same<T, float>::value) {
      if (x->tc && tc_gemm_eligible(g)) return tc_gemm(g, x->three, *x->w, s);
    } else {
      if (x->oz && oz_gemm_eligible(g)) return oz_gemm(g, *x->o, s);
    }
    return gemm_simt<T>(g, s, nullptr, 0);
  };
  QrGemm<T> qg, qg_side;
  qg.ctx = &ctx; qg.fn = fn;
  qg_side.ctx = &ctx_side; qg_side.fn = fn;
  return householder_qr<T>(static_cast<cx<T>*>(A), lda, m, n, static_cast<cx<T>*>(Q), ldq, qs, st,
                           device_error_word(), &qg, &qg_side);
}
__global__ void k_fill_unit(float2* x, long long n, unsigned seed) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  unsigned h = (unsigned)i * 2654435761u ^ seed;
  h ^= h >> 15; h *= 2246822519u; h ^= h >> 13;
  x[i] = make_float2((float)(h & 0xffff) / 32768.f - 1.f, (float)(h >> 16) / 32768.f - 1.f);
}
__global__ void k_fill_unit64(double2* x, long long n, unsigned seed) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  unsigned h = (unsigned)i * 2654435761u ^ seed;
  h ^= h >> 15; h *= 2246822519u; h ^= h >> 13;
  x[i] = make_double2((double)(h & 0xffff) / 32768.0 - 1.0, (double)(h >> 16) / 32768.0 - 1.0);
}
std::mutex g_tune_run_mu;  // one tuning pass at a time (the recording is process-wide)
}  // namespace
}  // namespace qrtebd

extern "C" {

int qrtebd_trunc_default(qrtebd_trunc* tr, int scheme, int chi_max) {
  if (!tr || chi_max < 1 || (scheme != QRTEBD_PLAIN && scheme != QRTEBD_CBE)) return QRTEBD_ERR_INVALID_ARG;
  tr->scheme = scheme;
  tr->chi_max = chi_max;
  tr->eta = 0;
  tr->dchi_min = 100;
  tr->dchi_frac = 0.1;
  tr->svd_min = 1e-14;
  tr->tie_tol = 1e-10;
  tr->eps_explicit = 0;
  tr->eps_target = 0.0;
  tr->reorth = -1;
  tr->sweeps = 1;
  return QRTEBD_OK;
}

int qrtebd_bond_workspace_size(int precision, int chi_l, int d, int chi_m, int chi_r, int xi_kind,
                               int theta_given, const qrtebd_trunc* tr, size_t* bytes) {
  if (!bytes || !tr) return QRTEBD_ERR_INVALID_ARG;
  qrtebd_bond_io io;
  std::memset(&io, 0, sizeof io);
  io.precision = precision;
  io.chi_l = chi_l; io.d = d; io.chi_m = chi_m; io.chi_r = chi_r;
  io.xi_kind = xi_kind;
  static const char dummy = 0;
  io.bm = theta_given ? nullptr : &dummy;
  return bond_update(&io, tr, nullptr, nullptr, bytes);
}

int qrtebd_bond_update(const qrtebd_bond_io* io, const qrtebd_trunc* tr, void* stream,
                       qrtebd_bond_info* info) {
  return bond_update(io, tr, static_cast<cudaStream_t>(stream), info, nullptr);
}


int qrtebd_autotune_bond(int precision, int chi_l, int d, int chi_m, int chi_r, int xi_kind,
                         int theta_given, const qrtebd_trunc* tr, void* stream, int* n_shapes) {
  if (!tr || chi_l < 1 || d < 1 || chi_m < 1 || chi_r < 1 || xi_kind < 0 || xi_kind > 3)
    return QRTEBD_ERR_INVALID_ARG;
  if (n_shapes) *n_shapes = 0;
  if (precision != QRTEBD_C64_3XTF32 && precision != QRTEBD_C64_TF32) return QRTEBD_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  size_t ws = 0;
  QR_TRY(qrtebd_bond_workspace_size(precision, chi_l, d, chi_m, chi_r, xi_kind, theta_given, tr, &ws));
  const long long eta = choose_eta(tr, chi_l, d, chi_m, chi_r);
  if (eta < 1) return QRTEBD_ERR_INVALID_ARG;
  const long long mL = (long long)chi_l * d, nR = (long long)d * chi_r;
  // synthetic operands of the bond's shape (values in [-1, 1]); one allocation
  const long long n_in[4] = {(xi_kind == 1 || xi_kind == 3) ? (long long)chi_l * chi_l : chi_l,
                             theta_given ? 0 : mL * chi_m, (long long)chi_m * nR,
                             theta_given ? mL * nR : 0};
  const long long n_out[3] = {mL * eta, eta * eta, eta * nR};
  const long long n_gate = (long long)d * d * d * d;  // complex128
  size_t off = 0;
  auto carve = [&](size_t bytes) { size_t o = off; off += align_up(bytes, 256); return o; };
  size_t o_in[4], o_out[3];
  for (int i = 0; i < 4; ++i) o_in[i] = carve((size_t)n_in[i] * sizeof(float2));
  for (int i = 0; i < 3; ++i) o_out[i] = carve((size_t)n_out[i] * sizeof(float2));
  const size_t o_gate = carve((size_t)n_gate * sizeof(double2));
  const size_t o_stats = carve(4 * sizeof(double));
  const size_t o_s = carve((size_t)eta * sizeof(double));
  const size_t o_ws = carve(ws);
  char* mem = nullptr;
  QR_CUDA_TRY(cudaMalloc(&mem, off));
  std::lock_guard<std::mutex> lk(g_tune_run_mu);
  int rc = QRTEBD_OK;
  std::vector<TcShape> shapes;
  do {
    for (int i = 0; i < 4; ++i)
      if (n_in[i] > 0)
        k_fill_unit<<<(unsigned)ceil_div(n_in[i], 256), 256, 0, st>>>(
            reinterpret_cast<float2*>(mem + o_in[i]), n_in[i], 17u + i);
    k_fill_unit64<<<(unsigned)ceil_div(n_gate, 256), 256, 0, st>>>(
        reinterpret_cast<double2*>(mem + o_gate), n_gate, 5u);
    if (cudaGetLastError() != cudaSuccess) { rc = QRTEBD_ERR_CUDA; break; }
    qrtebd_bond_io io;
    std::memset(&io, 0, sizeof io);
    io.precision = precision;
    io.chi_l = chi_l; io.d = d; io.chi_m = chi_m; io.chi_r = chi_r;
    io.xi_kind = xi_kind;
    io.xi = xi_kind ? mem + o_in[0] : nullptr;
    io.bm = theta_given ? nullptr : mem + o_in[1];
    io.bn = mem + o_in[2];
    io.theta = theta_given ? mem + o_in[3] : nullptr;
    io.gate = mem + o_gate;
    io.bm_out = mem + o_out[0]; io.xi_out = mem + o_out[1]; io.bn_out = mem + o_out[2];
    io.stats_out = reinterpret_cast<double*>(mem + o_stats);
    io.schmidt_out = reinterpret_cast<double*>(mem + o_s);
    io.workspace = mem + o_ws; io.workspace_bytes = ws;
    // pass 1: record the tensor-core product shapes of one update
    tc_record_begin();
    qrtebd_bond_info info;
    rc = bond_update(&io, tr, st, &info, nullptr);
    shapes = tc_record_end();
    if (rc != QRTEBD_OK) break;
    if (cudaStreamSynchronize(st) != cudaSuccess) { rc = QRTEBD_ERR_CUDA; break; }
  } while (false);
  cudaError_t fe = cudaStreamSynchronize(st);
  cudaFree(mem);
  if (rc != QRTEBD_OK) return rc;
  if (fe != cudaSuccess) { set_last_message(cudaGetErrorString(fe)); return QRTEBD_ERR_CUDA; }
  // pass 2: time the candidates of every shape not tuned yet
  int n = 0;
  for (const TcShape& sh : shapes) {
    TcConfig c;
    if (tc_tune_get(sh, &c)) continue;
    QR_TRY(tc_tune_shape(sh, st, nullptr));
    ++n;
  }
  if (n_shapes) *n_shapes = n;
  return QRTEBD_OK;
}

int qrtebd_autotune_count(void) { return (int)tc_tune_list().size(); }

int qrtebd_autotune_entry(int i, int shape[4], int config[3], double ms[2]) {
  const std::vector<TcTuned> v = tc_tune_list();
  if (i < 0 || i >= (int)v.size() || !shape || !config) return QRTEBD_ERR_INVALID_ARG;
  const TcTuned& t = v[i];
  shape[0] = t.shape.M; shape[1] = t.shape.N; shape[2] = t.shape.K; shape[3] = t.shape.three;
  config[0] = t.cfg.bn; config[1] = t.cfg.splits; config[2] = t.cfg.tail;
  if (ms) { ms[0] = t.ms_tuned; ms[1] = t.ms_default; }
  return QRTEBD_OK;
}

int qrtebd_autotune_set(const int shape[4], const int config[3]) {
  if (!shape || !config) return QRTEBD_ERR_INVALID_ARG;
  const TcShape s{shape[0], shape[1], shape[2], shape[3] ? 1 : 0};
  const TcConfig c{config[0], config[1], config[2] ? 1 : 0};
  if (s.M < s.N || s.N < 1 || s.K < 1 || (c.bn != 128 && c.bn != 256) || c.splits < 0 || c.splits > 32)
    return QRTEBD_ERR_INVALID_ARG;
  tc_tune_put(TcTuned{s, c, 0.0, 0.0});
  return QRTEBD_OK;
}

void qrtebd_autotune_clear(void) { tc_tune_clear(); }

int qrtebd_tc_operand_prep(int mode, int* previous) {
  if (mode != 0 && mode != 1) return QRTEBD_ERR_INVALID_ARG;
  const int prev = tc_prep_mode(mode);
  if (previous) *previous = prev;
  return QRTEBD_OK;
}

int qrtebd_stream_check(void* stream) { return check_device_error(static_cast<cudaStream_t>(stream)); }

int qrtebd_set_spin_limit(long long polls) {
  const long long v = polls <= 0 ? kSpinLimit : polls;
  std::lock_guard<std::mutex> lk(barrier_spin_mu());
  for (const void* sym : barrier_spin_symbols()) QR_CUDA_TRY(cudaMemcpyToSymbol(sym, &v, sizeof v));
  return QRTEBD_OK;
}

int qrtebd_selftest_barrier_timeout(void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned* err = device_error_word();
  if (!err) { set_last_message("device error word unavailable"); return QRTEBD_ERR_CUDA; }
  void* bar = nullptr;
  QR_CUDA_TRY(cudaGetSymbolAddress(&bar, g_selftest_bar));
  QR_CUDA_TRY(cudaMemsetAsync(bar, 0, sizeof(g_selftest_bar), st));
  k_selftest_barrier<<<1, 32, 0, st>>>(static_cast<unsigned*>(bar), err);
  note_launch();
  QR_CUDA_TRY(cudaGetLastError());
  return QRTEBD_OK;
}

int qrtebd_zgemm(int precision, int m, int n, int k, const void* A, long long sam, long long sak,
                 int conj_a, const void* B, long long sbk, long long sbn, int conj_b, void* C,
                 long long scm, long long scn, const double* alpha, const double* beta,
                 void* workspace, size_t workspace_bytes, void* stream) {
  if (m < 0 || n < 0 || k < 0 || !A || !B || !C || !alpha || !beta) return QRTEBD_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (prec_is_c128(precision)) {
    GemmArgs<double> g{m, n, k, static_cast<const double2*>(A), sam, sak, conj_a != 0,
                       static_cast<const double2*>(B), sbk, sbn, conj_b != 0,
                       static_cast<double2*>(C), scm, scn,
                       make_double2(alpha[0], alpha[1]), make_double2(beta[0], beta[1])};
    if (precision == QRTEBD_C128_OZ && m > 0 && n > 0 && k > 0 && oz_gemm_eligible(g)) {
      Arena ar;
      ar.base = static_cast<char*>(workspace);
      ar.cap = workspace_bytes;
      OzWorkspace w;
      oz_carve(ar, std::max(m, n), k, std::min(m, n), w);
      if (ar.overflow() || !workspace) { set_last_message("zgemm: workspace too small"); return QRTEBD_ERR_OOM; }
      return oz_gemm(g, w, st);
    }
    return gemm_simt<double>(g, st, nullptr, 0);
  }
  GemmArgs<float> g{m, n, k, static_cast<const float2*>(A), sam, sak, conj_a != 0,
                    static_cast<const float2*>(B), sbk, sbn, conj_b != 0,
                    static_cast<float2*>(C), scm, scn,
                    make_float2((float)alpha[0], (float)alpha[1]),
                    make_float2((float)beta[0], (float)beta[1])};
  if (precision == QRTEBD_C64_FP32) return gemm_simt<float>(g, st, nullptr, 0);
  if (precision != QRTEBD_C64_3XTF32 && precision != QRTEBD_C64_TF32) return QRTEBD_ERR_INVALID_ARG;
  if (m == 0 || n == 0) return QRTEBD_OK;
  if (k == 0) return gemm_simt<float>(g, st, nullptr, 0);  // C = beta C
  Arena ar;
  ar.base = static_cast<char*>(workspace);
  ar.cap = workspace_bytes;
  TcWorkspace w;
  tc_carve(ar, std::max(m, n), k, std::max(m, n), w);
  if (ar.overflow() || !workspace) { set_last_message("zgemm: workspace too small"); return QRTEBD_ERR_OOM; }
  return tc_gemm(g, precision == QRTEBD_C64_3XTF32, w, st);
}

size_t qrtebd_zgemm_workspace_size(int m, int n, int k) {
  Arena ar;
  ar.measuring = true;
  TcWorkspace w;
  tc_carve(ar, std::max(m, n), k, std::max(m, n), w);
  Arena ao;
  ao.measuring = true;
  OzWorkspace ow;
  oz_carve(ao, std::max(m, n), k, std::min(m, n), ow);
  return std::max(ar.off, ao.off);
}


int qrtebd_householder_qr(int precision, int m, int n, void* A, long long lda, void* Q,
                          long long ldq, void* workspace, size_t workspace_bytes, void* stream) {
  if (m < n || n < 1 || !A || !Q || lda < n || ldq < n) return QRTEBD_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (prec_is_c128(precision))
    return qr_entry<double>(precision, m, n, A, lda, Q, ldq, workspace, workspace_bytes, st, nullptr);
  if (!prec_valid(precision)) return QRTEBD_ERR_INVALID_ARG;
  return qr_entry<float>(precision, m, n, A, lda, Q, ldq, workspace, workspace_bytes, st, nullptr);
}

size_t qrtebd_qr_workspace_size(int precision, int m, int n) {
  size_t need = 0;
  if (m < n || n < 1) return 0;
  if (prec_is_c128(precision))
    qr_entry<double>(precision, m, n, nullptr, n, nullptr, n, nullptr, 0, nullptr, &need);
  else
    qr_entry<float>(precision, m, n, nullptr, n, nullptr, n, nullptr, 0, nullptr, &need);
  return need;
}

size_t qrtebd_cbe_decompose_workspace_size(int precision, int n) {
  if (n < 1) return 0;
  if (prec_is_c128(precision)) {
    if (svd64_supported(n)) return svd64_work_bytes(n);
    return (2 * (size_t)n * n + herm_eig_scratch_elems(n)) * sizeof(double2) +
           gemm_simt_scratch_elems(n, n, n, 1) * sizeof(double2) + 1024;
  }
  return svd32_work_bytes(n);
}

int qrtebd_cbe_decompose(int precision, int n, const void* Rz, long long ldr, double* w, void* Vh,
                         void* workspace, size_t workspace_bytes, int* sweeps, void* stream) {
  if (n < 1 || ldr < n || !Rz || !w || !Vh || !workspace) return QRTEBD_ERR_INVALID_ARG;
  if (!prec_valid(precision)) return QRTEBD_ERR_INVALID_ARG;
  if (workspace_bytes < qrtebd_cbe_decompose_workspace_size(precision, n)) return QRTEBD_ERR_OOM;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned* err = device_error_word();
  if (!prec_is_c128(precision))
    return svd_rows_jacobi32(static_cast<const float2*>(Rz), ldr, n, w, static_cast<double2*>(Vh),
                             workspace, workspace_bytes, st, err, sweeps);
  if (svd64_supported(n))
    return svd_rows_jacobi64(static_cast<const double2*>(Rz), ldr, n, w, static_cast<double2*>(Vh),
                             workspace, workspace_bytes, st, err, sweeps);
  // complex128 beyond the one-sided solver's shared memory: M = Rz Rz^dag (FP64), two-sided Jacobi
  const size_t nn = (size_t)n * n;
  double2* M = static_cast<double2*>(workspace);
  double2* M2 = M + nn;
  double2* scr = M2 + nn;
  const size_t se = herm_eig_scratch_elems(n);
  double2* gscr = scr + se;
  const double2* R = static_cast<const double2*>(Rz);
  GemmArgs<double> g{n, n, n, R, ldr, 1, false, R, 1, ldr, true, M, n, 1, make_double2(1, 0),
                     make_double2(0, 0)};
  QR_TRY(gemm_simt<double>(g, st, gscr, gemm_simt_scratch_elems(n, n, n, 1)));
  QR_TRY(herm_eig(M, n, w, static_cast<double2*>(Vh), scr, se, st, err));
  if (sweeps) QR_CUDA_TRY(cudaMemsetAsync(sweeps, 0, sizeof(int), st));
  (void)M2;
  return QRTEBD_OK;
}

int qrtebd_clock_bond_gate(int d, double g, double wl, double wr, double tau_re, double tau_im,
                           double* U_out) {
  if (d < 2 || d > 64 || !U_out) return QRTEBD_ERR_INVALID_ARG;
  const int n = d * d;
  const double pi = 3.14159265358979323846;
  std::vector<zc> Z(d), X((size_t)d * d, 0.0);
  for (int k = 0; k < d; ++k) Z[k] = std::polar(1.0, 2 * pi * k / d);
  for (int k = 0; k < d; ++k) X[(size_t)k * d + (k + 1) % d] = 1.0;
  std::vector<zc> Xs((size_t)d * d);
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) Xs[(size_t)i * d + j] = X[(size_t)i * d + j] + std::conj(X[(size_t)j * d + i]);
  std::vector<zc> h((size_t)n * n, 0.0);
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j)
      for (int k = 0; k < d; ++k)
        for (int l = 0; l < d; ++l) {
          zc v = 0;
          if (i == k && j == l) v -= Z[i] * std::conj(Z[j]) + std::conj(Z[i]) * Z[j];
          if (j == l) v -= g * wl * Xs[(size_t)i * d + k];
          if (i == k) v -= g * wr * Xs[(size_t)j * d + l];
          h[(size_t)(i * d + j) * n + (k * d + l)] = v;
        }
  std::vector<zc> V;
  std::vector<double> w;
  herm_jacobi_host(n, h, V, w);
  const zc tau(tau_re, tau_im), I(0, 1);
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) {
      zc s = 0;
      for (int k = 0; k < n; ++k) s += V[(size_t)r * n + k] * std::exp(-I * tau * w[k]) * std::conj(V[(size_t)c * n + k]);
      U_out[2 * ((size_t)r * n + c)] = s.real();
      U_out[2 * ((size_t)r * n + c) + 1] = s.imag();
    }
  return QRTEBD_OK;
}

int qrtebd_clock_bond_gate_charge(int d, double g, double wl, double wr, double tau_re,
                                  double tau_im, double* U_out) {
  if (d < 2 || d > 64 || !U_out) return QRTEBD_ERR_INVALID_ARG;
  const int n = d * d;
  std::vector<double> Uz(2 * (size_t)n * n);
  QR_TRY(qrtebd_clock_bond_gate(d, g, wl, wr, tau_re, tau_im, Uz.data()));
  const double pi = 3.14159265358979323846;
  // F2[(a b), (i j)] = F[a][i] F[b][j], F[a][i] = w^(a i) / sqrt(d)
  auto F = [&](int a, int i) { return std::polar(1.0 / std::sqrt((double)d), 2 * pi * ((a * i) % d) / d); };
  std::vector<zc> T((size_t)n * n);  // T = U F2
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) {
      zc s = 0;
      for (int k = 0; k < n; ++k)
        s += zc(Uz[2 * ((size_t)r * n + k)], Uz[2 * ((size_t)r * n + k) + 1]) * F(k / d, c / d) * F(k % d, c % d);
      T[(size_t)r * n + c] = s;
    }
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) {
      zc s = 0;
      if ((r / d + r % d) % d == (c / d + c % d) % d)
        for (int k = 0; k < n; ++k) s += std::conj(F(k / d, r / d) * F(k % d, r % d)) * T[(size_t)k * n + c];
      U_out[2 * ((size_t)r * n + c)] = s.real();
      U_out[2 * ((size_t)r * n + c) + 1] = s.imag();
    }
  return QRTEBD_OK;
}

const char* qrtebd_strerror(int status) {
  switch (status) {
    case QRTEBD_OK: return "ok";
    case QRTEBD_ERR_INVALID_ARG: return "invalid argument";
    case QRTEBD_ERR_OOM: return "out of memory";
    case QRTEBD_ERR_CUDA: return "CUDA error";
    case QRTEBD_ERR_TIMEOUT: return "bounded wait expired";
    case QRTEBD_ERR_NUMERIC: return "numerical error (NaN/Inf)";
    case QRTEBD_ERR_NOT_ADMITTED: return "not admitted";
    default: return "unknown status";
  }
}

const char* qrtebd_last_error_message(void) { return g_msg.c_str(); }

const char* qrtebd_version(void) { return "qrtebd 0.1 (sm_103a)"; }

}  // extern "C"
