// Generic strided complex GEMM on CUDA cores; see gemm_simt.cuh.
//
// 64x64 output tile per 256-thread block, 4x4 complex outputs per thread, K
// staged through shared memory in steps of 16. Loads pick the thread mapping
// along whichever index of the operand is contiguous, so row-major, transposed
// and conjugate-transposed operands are all read coalesced.
// Complex128 products with few 64x64 tiles run with 16x16 tiles instead (one output per
// thread): B300's FP64 pipe (~1.7 FMA per clock per SM) makes such a product bound by the
// FP64 work of its busiest SM, so it is spread over as many SMs as the output allows (a
// 96 x 96 x 32 product: 36 CTAs instead of 4).
#include "gemm_simt.cuh"

namespace qrtebd {

namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

template <typename T>
__global__ void __launch_bounds__(NT) k_gemm(GemmArgs<T> g, int ksplit, int kchunk,
                                             cx<T>* partial) {
  __shared__ cx<T> As[BK][BM + 1];
  __shared__ cx<T> Bs[BK][BN + 1];
  pdl_launch_dependents();
  pdl_wait();
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int bz = blockIdx.z / ksplit, sz = blockIdx.z % ksplit;
  const cx<T>* A = g.A + bz * g.bsa;
  const cx<T>* B = g.B + bz * g.bsb;
  const int kbeg = sz * kchunk;
  const int kend = min(g.K, kbeg + kchunk);
  const bool a_kc = (g.sak == 1);
  const bool b_nc = (g.sbn == 1);

  cx<T> acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = mk<T>(0, 0);

  for (int k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
    for (int r = 0; r < (BM * BK) / NT; ++r) {
      int l = tid + r * NT;
      int mm, kk;
      if (a_kc) { mm = l / BK; kk = l % BK; } else { mm = l % BM; kk = l / BM; }
      int gm = m0 + mm, gk = k0 + kk;
      cx<T> v = mk<T>(0, 0);
      if (gm < g.M && gk < kend) {
        v = A[gm * g.sam + gk * g.sak];
        if (g.conj_a) v.y = -v.y;
      }
      As[kk][mm] = v;
    }
#pragma unroll
    for (int r = 0; r < (BN * BK) / NT; ++r) {
      int l = tid + r * NT;
      int nn, kk;
      if (b_nc) { kk = l / BN; nn = l % BN; } else { nn = l / BK; kk = l % BK; }
      int gn = n0 + nn, gk = k0 + kk;
      cx<T> v = mk<T>(0, 0);
      if (gn < g.N && gk < kend) {
        v = B[gk * g.sbk + gn * g.sbn];
        if (g.conj_b) v.y = -v.y;
      }
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      cx<T> a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) cfma<T>(acc[i][j], a[i], b[j]);
    }
    __syncthreads();
  }

  if (ksplit > 1) {
    // raw partial sums, dense [batch][split][M][N]
    cx<T>* P = partial + ((long long)bz * ksplit + sz) * (long long)g.M * g.N;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        int gm = m0 + ty + 16 * i, gn = n0 + tx + 16 * j;
        if (gm < g.M && gn < g.N) P[(long long)gm * g.N + gn] = acc[i][j];
      }
    return;
  }
  cx<T>* C = g.C + bz * g.bsc;
  const bool use_beta = (g.beta.x != T(0) || g.beta.y != T(0));
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int gm = m0 + ty + 16 * i, gn = n0 + tx + 16 * j;
      if (gm < g.M && gn < g.N) {
        cx<T>* p = C + gm * g.scm + gn * g.scn;
        cx<T> v = cmul<T>(g.alpha, acc[i][j]);
        if (use_beta) v = cadd<T>(v, cmul<T>(g.beta, *p));
        *p = v;
      }
    }
}

template <typename T>
__global__ void k_splitk_reduce(GemmArgs<T> g, int ksplit, const cx<T>* partial) {
  pdl_launch_dependents();
  pdl_wait();
  long long MN = (long long)g.M * g.N;
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  int bz = blockIdx.y;
  if (idx >= MN) return;
  int gm = (int)(idx / g.N), gn = (int)(idx % g.N);
  const cx<T>* P = partial + (long long)bz * ksplit * MN;
  cx<T> s = mk<T>(0, 0);
  for (int z = 0; z < ksplit; ++z) s = cadd<T>(s, P[z * MN + idx]);
  cx<T>* p = g.C + bz * g.bsc + gm * g.scm + gn * g.scn;
  cx<T> v = cmul<T>(g.alpha, s);
  if (g.beta.x != T(0) || g.beta.y != T(0)) v = cadd<T>(v, cmul<T>(g.beta, *p));
  *p = v;
}

constexpr int SB = 16;  // small tile (complex128 products with few 64x64 tiles)

template <typename T>
__global__ void __launch_bounds__(SB * SB) k_gemm_small(GemmArgs<T> g, int ksplit, int kchunk,
                                                       cx<T>* partial) {
  __shared__ cx<T> As[SB][SB + 1];
  __shared__ cx<T> Bs[SB][SB + 1];
  pdl_launch_dependents();
  pdl_wait();
  const int tid = threadIdx.x;
  const int tx = tid % SB, ty = tid / SB;  // output column, row
  const int m0 = blockIdx.y * SB, n0 = blockIdx.x * SB;
  const int bz = blockIdx.z / ksplit, sz = blockIdx.z % ksplit;
  const cx<T>* A = g.A + bz * g.bsa;
  const cx<T>* B = g.B + bz * g.bsb;
  const int kbeg = sz * kchunk;
  const int kend = min(g.K, kbeg + kchunk);
  const bool a_kc = (g.sak == 1);
  const bool b_nc = (g.sbn == 1);
  cx<T> acc0 = mk<T>(0, 0), acc1 = mk<T>(0, 0);
  for (int k0 = kbeg; k0 < kend; k0 += SB) {
    {
      const int mm = a_kc ? tid / SB : tid % SB, kk = a_kc ? tid % SB : tid / SB;
      const int gm = m0 + mm, gk = k0 + kk;
      cx<T> v = mk<T>(0, 0);
      if (gm < g.M && gk < kend) {
        v = A[gm * g.sam + gk * g.sak];
        if (g.conj_a) v.y = -v.y;
      }
      As[kk][mm] = v;
    }
    {
      const int kk = b_nc ? tid / SB : tid % SB, nn = b_nc ? tid % SB : tid / SB;
      const int gn = n0 + nn, gk = k0 + kk;
      cx<T> v = mk<T>(0, 0);
      if (gn < g.N && gk < kend) {
        v = B[gk * g.sbk + gn * g.sbn];
        if (g.conj_b) v.y = -v.y;
      }
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < SB; kk += 2) {
      cfma<T>(acc0, As[kk][ty], Bs[kk][tx]);
      cfma<T>(acc1, As[kk + 1][ty], Bs[kk + 1][tx]);
    }
    __syncthreads();
  }
  const cx<T> acc = cadd<T>(acc0, acc1);
  const int gm = m0 + ty, gn = n0 + tx;
  if (gm >= g.M || gn >= g.N) return;
  if (ksplit > 1) {
    partial[((long long)bz * ksplit + sz) * (long long)g.M * g.N + (long long)gm * g.N + gn] = acc;
    return;
  }
  cx<T>* p = g.C + bz * g.bsc + gm * g.scm + gn * g.scn;
  cx<T> v = cmul<T>(g.alpha, acc);
  if (g.beta.x != T(0) || g.beta.y != T(0)) v = cadd<T>(v, cmul<T>(g.beta, *p));
  *p = v;
}

// the small-tile form: complex128 products with fewer than 64 tiles of 64 x 64
bool use_small(int M, int N, int batch) {
  return ceil_div(M, BM) * ceil_div(N, BN) * (long long)batch < 64;
}
int pick_ksplit_small(int M, int N, int K, int batch) {
  const long long tiles = ceil_div(M, SB) * ceil_div(N, SB) * (long long)batch;
  if (tiles >= 148 || K < 4 * SB) return 1;
  const long long want = ceil_div(2 * 148, tiles), maxs = K / (2 * SB);
  const int s = (int)std::min<long long>(std::min<long long>(want, maxs), 64);
  return s < 1 ? 1 : s;
}

int pick_ksplit(int M, int N, int K, int batch) {
  long long tiles = ceil_div(M, BM) * ceil_div(N, BN) * (long long)batch;
  if (tiles >= 148 || K < 4 * BK) return 1;
  long long want = ceil_div(2 * 148, tiles);
  long long maxs = K / (2 * BK);
  int s = (int)std::min<long long>(std::min<long long>(want, maxs), 64);
  return s < 1 ? 1 : s;
}

}  // namespace

size_t gemm_simt_scratch_elems(int M, int N, int K, int batch) {
  int s = pick_ksplit(M, N, K, batch);
  if (use_small(M, N, batch)) s = std::max(s, pick_ksplit_small(M, N, K, batch));  // complex128 form
  return s > 1 ? (size_t)s * M * N * batch : 0;
}

template <typename T>
int gemm_simt(const GemmArgs<T>& g, cudaStream_t st, cx<T>* scratch, size_t scratch_elems,
              int prof_family) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return QRTEBD_OK;
  if (g.K <= 0) {
    // C = beta C: run with K = 0 through the normal path (acc stays zero)
  }
  const bool small = std::is_same<T, double>::value && use_small(g.M, g.N, g.batch);
  const int tm = small ? SB : BM, tn = small ? SB : BN;
  int ks = small ? pick_ksplit_small(g.M, g.N, g.K, g.batch) : pick_ksplit(g.M, g.N, g.K, g.batch);
  if (ks > 1 && (scratch == nullptr || scratch_elems < (size_t)ks * g.M * g.N * g.batch)) ks = 1;
  int kchunk = ks > 1 ? (int)(ceil_div(ceil_div(g.K, ks), BK) * BK) : (g.K > 0 ? g.K : 1);
  if (ks > 1) ks = (int)ceil_div(g.K, kchunk);
  dim3 grid((unsigned)ceil_div(g.N, tn), (unsigned)ceil_div(g.M, tm), (unsigned)(g.batch * ks));
  if (grid.y > 65535 || grid.z > 65535) return QRTEBD_ERR_INVALID_ARG;
  ProfScope prof(prof_family, st, 8.0 * g.M * g.N * (double)g.K * g.batch);
  if (small) QR_CUDA_TRY(launch_pdl(k_gemm_small<T>, grid, dim3(SB * SB), 0, st, g, ks, kchunk, scratch));
  else QR_CUDA_TRY(launch_pdl(k_gemm<T>, grid, dim3(NT), 0, st, g, ks, kchunk, scratch));
  note_launch();
  QR_CUDA_TRY(cudaGetLastError());
  if (ks > 1) {
    long long MN = (long long)g.M * g.N;
    dim3 rg((unsigned)ceil_div(MN, 256), (unsigned)g.batch);
    QR_CUDA_TRY(launch_pdl(k_splitk_reduce<T>, rg, dim3(256), 0, st, g, ks,
                           static_cast<const cx<T>*>(scratch)));
    note_launch();
    QR_CUDA_TRY(cudaGetLastError());
  }
  return QRTEBD_OK;
}

template int gemm_simt<float>(const GemmArgs<float>&, cudaStream_t, float2*, size_t, int);
template int gemm_simt<double>(const GemmArgs<double>&, cudaStream_t, double2*, size_t, int);

}  // namespace qrtebd
