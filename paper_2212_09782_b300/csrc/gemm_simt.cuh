// Generic strided complex GEMM on CUDA cores (FP32 or FP64 arithmetic).
//
//   C[m, n] = alpha * sum_k opA(m, k) opB(k, n) + beta * C[m, n]
//   opA(m, k) = A[m*sam + k*sak] (conjugated if conj_a), opB likewise.
//
// Any transpose / conjugate-transpose of a row-major operand is a choice of
// strides, so one kernel serves every contraction of the bond update in
// complex128 and every small contraction in complex64.
#pragma once
#include "common.cuh"

namespace qrtebd {

template <typename T> struct GemmArgs {
  int M, N, K;
  const cx<T>* A; long long sam, sak; bool conj_a;
  const cx<T>* B; long long sbk, sbn; bool conj_b;
  cx<T>* C; long long scm, scn;
  cx<T> alpha, beta;
  int batch = 1;
  long long bsa = 0, bsb = 0, bsc = 0;  // batch strides (elements)
  // tensor-core path only: A is unchanged since an earlier call with the same
  // pointer, strides and shape in this workspace, so its prepared operand may be reused
  bool reuse_a = false;
  // tensor-core path only: A is lower triangular (A[m][k] = 0 for k > m, zeros stored), so
  // a tile of rows may stop its K loop after its last row; other paths read the zeros
  bool tri_a = false;
  // tensor-core path only: B is upper triangular (B[k][n] = 0 for k > n, zeros stored), so
  // a tile of columns may stop its K loop after its last column
  bool tri_b = false;
};

// Enqueue the GEMM. `scratch` (may be null) lets the launcher split K for
// short-wide outputs; scratch_elems is its capacity in complex elements.
template <typename T>
int gemm_simt(const GemmArgs<T>& g, cudaStream_t st, cx<T>* scratch = nullptr,
              size_t scratch_elems = 0, int prof_family = PROF_SIMT_GEMM);

// Scratch (complex elements) gemm_simt would like for split-K at these sizes.
size_t gemm_simt_scratch_elems(int M, int N, int K, int batch);

}  // namespace qrtebd
