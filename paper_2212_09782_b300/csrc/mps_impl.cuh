// Internals of the device-resident MPS shared by mps.cu and layer.cu.
#pragma once
#include <vector>

#include "bond.cuh"

struct qrtebd_mps {
  int L = 0, d = 0, infinite = 0, chi_max = 0, precision = 0;
  cudaStream_t st = nullptr;
  int nbonds_store = 0;           // finite: L+1, uniform: L
  std::vector<int> chi, cap;      // per stored bond
  std::vector<void*> B;           // per site, capacity cap[m] * d * cap[m+1]
  std::vector<void*> Xi;          // per bond, dense cap x cap
  std::vector<void*> xiv;         // per bond, diagonal vector (valid if xi_diag)
  std::vector<char> xi_diag;
  // per bond: Xi is lower triangular with its zeros stored (the L / ||L|| of a plain update),
  // so the product Xi theta~' skips the blocks above the diagonal; not saved in checkpoints
  std::vector<char> xi_lower;
  std::vector<char> chi_pending;  // CBE cut of this bond still on the device (stats slot of its gate)
  double* eps_acc = nullptr;      // per bond, device
  double* stats = nullptr;        // device double[4 * ngates]: one slot per gate bond
  double* layer_eps = nullptr;    // device, per gate bond
  double2* gates = nullptr;       // device, ngates * d^4
  void* ws = nullptr;
  size_t ws_bytes = 0;
  void* aux = nullptr;            // expectation / schmidt scratch
  size_t aux_bytes = 0;
  size_t esz = 0;                 // bytes per complex element
};

namespace qrtebd {
int mps_gate_count(const qrtebd_mps* s);
// Copy the gates of the bonds of `parity` to the device (on the state's stream).
int mps_upload_gates(qrtebd_mps* s, int parity, const double* gates_host);
// Workspace the update of bond (m, m+1) needs with the current bond dimensions.
int mps_bond_ws_need(const qrtebd_mps* s, int m, const qrtebd_trunc* tr, size_t* need);
// Update bond (m, m+1) in place on stream `st` with the given workspace; records its
// eps into layer_eps[m] and adds it to the bond's accumulated eps.
int mps_update_bond(qrtebd_mps* s, int m, const qrtebd_trunc* tr, cudaStream_t st, void* ws,
                    size_t ws_bytes);
// Read back the CBE cuts of the bonds updated since the last call (their stats slots; one
// synchronisation of the state's stream) into the host bond dimensions.
int mps_collect_cuts(qrtebd_mps* s);
// Drop every captured layer graph that references this state (before it is freed).
void executor_forget_state(qrtebd_mps* s);
}  // namespace qrtebd
