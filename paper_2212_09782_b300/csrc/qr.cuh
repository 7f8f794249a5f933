// Blocked Householder QR with explicit Q (the QR of Sec. II step (i) and the LQ
// of step (ii), which is the QR of Y^dag).
#pragma once
#include "common.cuh"
#include "gemm_simt.cuh"

namespace qrtebd {

// Contraction back-end for the block-reflector updates. The default runs the
// CUDA-core GEMM; the complex64 tensor-core path installs its own.
template <typename T> struct QrGemm {
  // returns status; same semantics as gemm_simt
  int (*fn)(const GemmArgs<T>& g, cudaStream_t st, void* ctx) = nullptr;
  void* ctx = nullptr;
};

template <typename T> struct QrScratch {
  cx<T>* V = nullptr;      // m x n explicit reflectors (unit lower trapezoidal per panel)
  cx<T>* tau = nullptr;    // n
  cx<T>* VT = nullptr;     // m x n: V T of every outer block (trailing updates, explicit Q)
  cx<T>* Tf = nullptr;     // ceil(n/nb) blocks of nb x nb triangular factors
  cx<T>* W = nullptr;      // nb x n
  cx<T>* W2 = nullptr;     // nb x n
  cx<T>* W2s = nullptr;    // W2 of the look-ahead (side-stream) updates
  cx<T>* G = nullptr;      // outer-block Gram matrix V^dag V
  cx<T>* Tall = nullptr;   // n x n compact-WY factor of the whole QR (complex64 with look-ahead)
  cx<T>* Cb = nullptr;     // n x nbo: V[:, 0:k]^dag V_b, then times T_b, for T_all's block columns
  cx<T>* Xb = nullptr;
  cx<T>* Wq = nullptr;     // n x n: T_all V_top^dag for the explicit Q
  cx<T>* wy_part = nullptr;  // fused narrow update: per-CTA partials of V^dag C
  cx<T>* wy_W = nullptr;     // and their sum
  cx<T>* pg = nullptr;       // complex128 grid panel: per-CTA partial sums, [2][148][33]
  unsigned* bar = nullptr;   // grid-barrier counter and generation
  cx<T>* gemm_scratch = nullptr;
  size_t gemm_scratch_elems = 0;
};

// Panel width used for an m x n factorisation.
int qr_panel_width(int m, int n, int elem_bytes);

// Carve the scratch for an m x n QR out of `ar` (size query when ar.measuring).
template <typename T> void qr_carve(Arena& ar, int m, int n, QrScratch<T>& s);

// A (m x n, m >= n, row-major with leading dimension lda) is overwritten: its
// upper n x n triangle holds R (real diagonal, LAPACK geqrf sign convention) and
// everything below is zeroed. Q (m x n, leading dimension ldq) receives the
// explicit isometry with A_in = Q R. err: device error word.
// side_gemm (optional, with its own workspaces): runs the part of each outer trailing
// update beyond the next outer block on a library-owned side stream (look-ahead), so the
// next block's panel chain starts as soon as its own columns are updated.
template <typename T>
int householder_qr(cx<T>* A, long long lda, int m, int n, cx<T>* Q, long long ldq,
                   QrScratch<T>& s, cudaStream_t st, unsigned* err,
                   const QrGemm<T>* gemm = nullptr, const QrGemm<T>* side_gemm = nullptr);

}  // namespace qrtebd
