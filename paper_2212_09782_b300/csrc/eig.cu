// Hermitian eigensolver for CBE step (iv) (Sec. III: diagonalise L^dag L = V^dag S^2 V).
//
// Parallel cyclic Jacobi in FP64 with the round-robin (circle) ordering: each
// of the n'-1 steps of a sweep (n' = n rounded up to even) rotates n'/2
// disjoint index pairs at once. A rotation G on (p, q), with a_pq = |a| e,
//   G = [[c, s e], [-s conj(e), c]],  t = tan(theta) = sign(z) / (|z| + sqrt(1 + z^2)),
//   z = (a_qq - a_pp) / (2 |a|),  c = 1 / sqrt(1 + t^2),  s = t c,
// zeroes (G^dag A G)_pq. Sweeps repeat until the off-diagonal Frobenius norm is
// below 1e-15 of the total (checked on the host once per sweep).
#include "bond.cuh"

namespace qrtebd {

namespace {

struct Rot { int p, q; double c; double sr, si; };  // s * e

__device__ __forceinline__ void pair_of(int r, int k, int np, int& p, int& q) {
  const int m = np - 1;
  if (k == 0) { p = r % m; q = m; }
  else { p = (r + k) % m; q = (r - k + m) % m; }
  if (p > q) { int t = p; p = q; q = t; }
}

__global__ void k_jac_rot(const double2* A, int n, int np, int r, Rot* rot) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= np / 2) return;
  int p, q;
  pair_of(r, k, np, p, q);
  Rot R{p, q, 1.0, 0.0, 0.0};
  if (q < n) {
    double2 apq = A[(long long)p * n + q];
    double ab = sqrt(apq.x * apq.x + apq.y * apq.y);
    double app = A[(long long)p * n + p].x, aqq = A[(long long)q * n + q].x;
    if (ab > 1e-300 && ab > 1e-18 * sqrt(fabs(app * aqq))) {
      double z = (aqq - app) / (2.0 * ab);
      double t = (z >= 0 ? 1.0 : -1.0) / (fabs(z) + sqrt(1.0 + z * z));
      double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
      R.c = c; R.sr = s * apq.x / ab; R.si = s * apq.y / ab;
    }
  } else {
    R.q = -1;
  }
  rot[k] = R;
}

// A <- A G (columns p, q) and V <- V G, for every row i
__global__ void k_jac_cols(double2* A, double2* V, int n, int np, const Rot* rot) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long tot = (long long)n * (np / 2);
  if (idx >= tot) return;
  int k = (int)(idx / n), i = (int)(idx % n);
  Rot R = rot[k];
  if (R.q < 0 || (R.sr == 0.0 && R.si == 0.0)) return;
  const double c = R.c, er = R.sr, ei = R.si;  // s e
  double2* mats[2] = {A, V};
  for (int w = 0; w < 2; ++w) {
    double2* M = mats[w];
    double2 x = M[(long long)i * n + R.p], y = M[(long long)i * n + R.q];
    // col_p' = c x - conj(s e) y ; col_q' = (s e) x + c y
    double2 np_, nq_;
    np_.x = c * x.x - (er * y.x + ei * y.y);
    np_.y = c * x.y - (er * y.y - ei * y.x);
    nq_.x = (er * x.x - ei * x.y) + c * y.x;
    nq_.y = (er * x.y + ei * x.x) + c * y.y;
    M[(long long)i * n + R.p] = np_;
    M[(long long)i * n + R.q] = nq_;
  }
}

// A <- G^dag A (rows p, q), for every column j
__global__ void k_jac_rows(double2* A, int n, int np, const Rot* rot) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long tot = (long long)n * (np / 2);
  if (idx >= tot) return;
  int k = (int)(idx / n), j = (int)(idx % n);
  Rot R = rot[k];
  if (R.q < 0 || (R.sr == 0.0 && R.si == 0.0)) return;
  const double c = R.c, er = R.sr, ei = R.si;
  double2 x = A[(long long)R.p * n + j], y = A[(long long)R.q * n + j];
  // row_p' = c x - (s e) y ; row_q' = conj(s e) x + c y
  double2 np_, nq_;
  np_.x = c * x.x - (er * y.x - ei * y.y);
  np_.y = c * x.y - (er * y.y + ei * y.x);
  nq_.x = (er * x.x + ei * x.y) + c * y.x;
  nq_.y = (er * x.y - ei * x.x) + c * y.y;
  A[(long long)R.p * n + j] = np_;
  A[(long long)R.q * n + j] = nq_;
}

__global__ void k_eye64(double2* V, int n) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)n * n) return;
  V[idx] = make_double2((idx / n) == (idx % n) ? 1.0 : 0.0, 0.0);
}

// off-diagonal and total squared Frobenius norms (single block, deterministic)
__global__ void k_offnorm(const double2* A, int n, double* out) {
  __shared__ double so[32], st[32];
  double off = 0, tot = 0;
  for (long long i = threadIdx.x; i < (long long)n * n; i += blockDim.x) {
    double2 v = A[i];
    double a2 = v.x * v.x + v.y * v.y;
    tot += a2;
    if (i / n != i % n) off += a2;
  }
  for (int o = 16; o > 0; o >>= 1) {
    off += __shfl_xor_sync(0xffffffffu, off, o);
    tot += __shfl_xor_sync(0xffffffffu, tot, o);
  }
  if ((threadIdx.x & 31) == 0) { so[threadIdx.x >> 5] = off; st[threadIdx.x >> 5] = tot; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a += so[w]; b += st[w]; }
    out[0] = a; out[1] = b;
  }
}

// eigenvalues = diag(A), sorted descending (stable selection by rank); Vh = rows of
// conj(V) in that order
__global__ void k_sort_out(const double2* A, const double2* V, int n, double* w, double2* Vh) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double li = A[(long long)i * n + i].x;
  int rank = 0;
  for (int j = 0; j < n; ++j) {
    double lj = A[(long long)j * n + j].x;
    if (lj > li || (lj == li && j < i)) ++rank;
  }
  w[rank] = li;
  for (int r = 0; r < n; ++r) {
    double2 v = V[(long long)r * n + i];
    Vh[(long long)rank * n + r] = make_double2(v.x, -v.y);
  }
}

}  // namespace

size_t herm_eig_scratch_elems(int n) {
  // V (n x n) + rotations (n/2+1 Rot = 40 B each, in double2 units) + 2 doubles
  return (size_t)n * n + (size_t)(n / 2 + 1) * 3 + 2;
}

int herm_eig(double2* A, int n, double* w, double2* Vh, double2* scratch, size_t scratch_elems,
             cudaStream_t st, unsigned* err) {
  (void)err;
  if (n < 1 || scratch_elems < herm_eig_scratch_elems(n)) return QRTEBD_ERR_INVALID_ARG;
  double2* V = scratch;
  Rot* rot = reinterpret_cast<Rot*>(scratch + (size_t)n * n);
  double* nrm = reinterpret_cast<double*>(scratch + (size_t)n * n + (size_t)(n / 2 + 1) * 3);
  const int np = (n % 2) ? n + 1 : n;
  long long nn = (long long)n * n;
  k_eye64<<<(unsigned)ceil_div(nn, 256), 256, 0, st>>>(V, n);
  note_launch();
  QR_CUDA_TRY(cudaGetLastError());
  if (n > 1) {
    const long long work = (long long)n * (np / 2);
    const unsigned gw = (unsigned)ceil_div(work, 256);
    const unsigned gr = (unsigned)ceil_div(np / 2, 128);
    double hn[2] = {0, 0};
    for (int sweep = 0; sweep < 30; ++sweep) {
      k_offnorm<<<1, 1024, 0, st>>>(A, n, nrm);
      note_launch();
      QR_CUDA_TRY(cudaGetLastError());
      QR_CUDA_TRY(cudaMemcpyAsync(hn, nrm, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
      QR_CUDA_TRY(cudaStreamSynchronize(st));
      if (!(hn[1] > 0) || hn[0] <= 1e-30 * hn[1]) break;
      for (int r = 0; r < np - 1; ++r) {
        k_jac_rot<<<gr, 128, 0, st>>>(A, n, np, r, rot);
        note_launch();
        k_jac_cols<<<gw, 256, 0, st>>>(A, V, n, np, rot);
        note_launch();
        k_jac_rows<<<gw, 256, 0, st>>>(A, n, np, rot);
        note_launch();
      }
      QR_CUDA_TRY(cudaGetLastError());
    }
  }
  k_sort_out<<<(unsigned)ceil_div(n, 128), 128, 0, st>>>(A, V, n, w, Vh);
  note_launch();
  QR_CUDA_TRY(cudaGetLastError());
  return QRTEBD_OK;
}

}  // namespace qrtebd
