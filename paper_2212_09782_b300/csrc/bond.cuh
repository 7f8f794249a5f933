// One QR-TEBD bond update on the device (Sec. II, Sec. III).
#pragma once
#include "common.cuh"
#include "gemm_simt.cuh"
#include "qr.cuh"

namespace qrtebd {

// Shared implementation of qrtebd_bond_workspace_size / qrtebd_bond_update:
// with bytes != nullptr only the workspace is measured (no GPU work).
int bond_update(const qrtebd_bond_io* io, const qrtebd_trunc* tr, cudaStream_t st,
                qrtebd_bond_info* info, size_t* bytes);

// Effective eta for these sizes (the policy of qrtebd_trunc).
int choose_eta(const qrtebd_trunc* tr, int chi_l, int d, int chi_m, int chi_r);

// Hermitian eigensolver used by CBE (cyclic Jacobi, FP64): A (n x n, device,
// row-major, Hermitian) is destroyed; w (device, n) receives the eigenvalues in
// DESCENDING order and Vh (device, n x n) the conjugated eigenvectors as rows, so
// that A = Vh^dag diag(w) Vh.
int herm_eig(double2* A, int n, double* w, double2* Vh, double2* scratch, size_t scratch_elems,
             cudaStream_t st, unsigned* err);
size_t herm_eig_scratch_elems(int n);

}  // namespace qrtebd
