// One QR-TEBD bond update on the device (Sec. II, Sec. III).
#pragma once
#include "common.cuh"
#include "gemm_simt.cuh"
#include "qr.cuh"

namespace qrtebd {

// Shared implementation of qrtebd_bond_workspace_size / qrtebd_bond_update:
// with bytes != nullptr only the workspace is measured (no GPU work).
// CBE: the cut chi~ stays on the device (stats_out[3], as a double) and every kernel after the
// cut reads it there; sync_chi = true reads it back at the end (one stream synchronisation) into
// info->chi_new, sync_chi = false leaves info->chi_new = -1 for the caller to collect later
// (no synchronisation: a CBE update can then be recorded into a CUDA graph).
// theta_gated = true: io->theta holds theta~' = U theta' (the gate already applied; io->gate
// is not read and d may be 1), as for the blocks of a charge-conserving update.
int bond_update(const qrtebd_bond_io* io, const qrtebd_trunc* tr, cudaStream_t st,
                qrtebd_bond_info* info, size_t* bytes, bool sync_chi = true,
                bool theta_gated = false);

// Effective eta for these sizes (the policy of qrtebd_trunc).
int choose_eta(const qrtebd_trunc* tr, int chi_l, int d, int chi_m, int chi_r);

// Hermitian eigensolver used by CBE (cyclic Jacobi, FP64): A (n x n, device,
// row-major, Hermitian) is destroyed; w (device, n) receives the eigenvalues in
// DESCENDING order and Vh (device, n x n) the conjugated eigenvectors as rows, so
// that A = Vh^dag diag(w) Vh.
int herm_eig(double2* A, int n, double* w, double2* Vh, double2* scratch, size_t scratch_elems,
             cudaStream_t st, unsigned* err);
size_t herm_eig_scratch_elems(int n);

// The CBE decomposition for complex64 (one-sided Jacobi, FP32 rows, FP64 rotation
// parameters): Rz (n x n, device, row-major, leading dimension ldr) is read; w (device, n)
// receives the eigenvalues of Rz Rz^dag = L^dag L (the squared singular values of L, FP64)
// in DESCENDING order and Vh (device, n x n) the conjugated eigenvectors as rows, with the
// contract of herm_eig. work: device, svd32_work_bytes(n). sweeps (optional, device int):
// sweeps run (SJ_MAX_SWEEPS + 1 = 41: stopped unconverged). One cooperative launch.
size_t svd32_work_bytes(int n);
// The same one-sided Jacobi for complex128 (FP64 rows, sums and rotations; one cooperative
// launch, no host synchronisation): the CBE decomposition of record for complex128 whenever
// svd64_supported(n) (a block pair of rows fits shared memory: n up to ~6800).
bool svd64_supported(int n);
size_t svd64_work_bytes(int n);
int svd_rows_jacobi64(const double2* Rz, long long ldr, int n, double* w, double2* Vh, void* work,
                      size_t work_bytes, cudaStream_t st, unsigned* err, int* sweeps = nullptr);
int svd_rows_jacobi32(const float2* Rz, long long ldr, int n, double* w, double2* Vh, void* work,
                      size_t work_bytes, cudaStream_t st, unsigned* err, int* sweeps = nullptr);

}  // namespace qrtebd
