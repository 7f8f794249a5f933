/*
 * qrtebd.h - C ABI of libqrtebd: the QR-based TEBD bond update on one B300 GPU.
 *
 * Method: Unfried, Hauschild, Pollmann, "Fast Time-Evolution of Matrix-Product
 * States using the QR decomposition", arXiv:2212.09782.
 *   - Sec. II, Fig. 2b steps (i)-(iii): the plain QR truncation.
 *   - Sec. III, Fig. 3 steps (i)-(v): QR with controlled bond expansion (CBE).
 *   - Sec. IV, Eqs. 2-3: the d-state clock model used as the workload.
 *
 * Conventions shared by every call:
 *   - Complex numbers are interleaved (re, im): complex128 = 2 doubles,
 *     complex64 = 2 floats. Every tensor is row-major, left index slowest.
 *   - Site tensor B (chi_l, d, chi_r); bond matrix Xi (chi, chi); the two-site
 *     block theta (chi_l, d, d, chi_r) is read as the (chi_l d) x (d chi_r)
 *     matrix with row alpha*d + i and column j*chi_r + delta.
 *   - A two-site gate U is a d^2 x d^2 complex128 matrix, row = output (i, j),
 *     column = input (i', j'), combined index i*d + j (left site most significant).
 *   - "device" pointers are CUDA device memory of the current device; "host"
 *     pointers are ordinary host memory. The caller owns every pointer it passes;
 *     the library never frees caller memory and keeps no pointer past the call.
 *   - Streams are passed as void* (a cudaStream_t); NULL is the legacy default stream.
 *   - Every call returns a status code (0 = OK, negative = error). No C++
 *     exception crosses this boundary. qrtebd_last_error_message() describes the
 *     most recent failure of the calling thread.
 */
#ifndef QRTEBD_H
#define QRTEBD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */
#define QRTEBD_OK 0
#define QRTEBD_ERR_INVALID_ARG (-1)  /* bad size, eta > d*chi, NULL where required */
#define QRTEBD_ERR_OOM (-2)          /* workspace too small or device allocation failed */
#define QRTEBD_ERR_CUDA (-3)         /* a CUDA runtime call failed */
#define QRTEBD_ERR_TIMEOUT (-4)      /* a kernel gave up a bounded wait */
#define QRTEBD_ERR_NUMERIC (-5)      /* NaN/Inf met in a norm */
#define QRTEBD_ERR_NOT_ADMITTED (-6) /* a request does not fit the memory budget */

/* -------------------------------------------------------------- precision */
/* Arithmetic of the bond update.
 *   C128       complex128 tensors, FP64 arithmetic everywhere.
 *   C64_3XTF32 complex64 tensors; the large contractions run on tcgen05 tensor
 *              cores as three TF32 products (hi*hi + hi*lo + lo*hi) with FP32
 *              accumulation; Householder norms and all reductions in FP64.
 *   C64_TF32   as C64_3XTF32 with one TF32 product (about 1e-3 relative error).
 *   C64_FP32   complex64 tensors, FP32 CUDA-core arithmetic (no tensor cores).
 *   C128_OZ    complex128 tensors; the large complex products run as FP64 emulated on the
 *              TF32 tensor cores (Ozaki splitting: every row scaled by a power of two and cut
 *              into 8 integer slices of 7 bits, the slice products summed exactly in FP32
 *              over 1024 terms and accumulated in FP64), about 1e-15 relative to the exact
 *              product; panels, norms and small products stay in FP64 on CUDA cores. */
#define QRTEBD_C128 0
#define QRTEBD_C64_3XTF32 1
#define QRTEBD_C64_TF32 2
#define QRTEBD_C64_FP32 3
#define QRTEBD_C128_OZ 4

/* -------------------------------------------------------------- truncation */
#define QRTEBD_PLAIN 0 /* Sec. II: eta fixed a priori, Xi~ = L (non-diagonal) */
#define QRTEBD_CBE 1   /* Sec. III: expand to eta, cut on the Schmidt values of L */

typedef struct qrtebd_trunc {
  int scheme;       /* QRTEBD_PLAIN or QRTEBD_CBE */
  int chi_max;      /* largest bond dimension kept (>= 1) */
  int eta;          /* > 0: use this expansion dimension; 0: the policy below */
  int dchi_min;     /* CBE: dchi = max(dchi_min, ceil(dchi_frac * chi_m)) (Fig. 4: 100) */
  double dchi_frac; /* CBE: relative expansion per update (Sec. III: about 0.1) */
  double svd_min;   /* CBE: drop Schmidt values below svd_min * ||S|| (Fig. 4: 1e-14) */
  double tie_tol;   /* CBE: never cut inside a multiplet closer than tie_tol * S_1 */
  int eps_explicit; /* 0: eps = 1 - kept / ||theta~||^2 (FP64 norms; exact for the orthogonal
                       projections of Sec. II, but with a floor of about the storage precision,
                       ~1e-7 in complex64); 1: eps from the explicit residual
                       ||theta~ - approx||^2 (one more contraction; the distance of Sec. IV) */
  double eps_target;  /* CBE: > 0 keeps the fewest Schmidt values whose discarded weight,
                         sum_{k > chi~} S_k^2 / sum_k S_k^2, is at most eps_target (within the
                         chi_max and svd_min cut, before the tie rule); 0: off. Plain: ignored
                         (its bond dimension is eta). */
  int reorth;         /* one re-orthogonalisation pass of the right isometry after the LQ
                         (both schemes): D = Q^dag Q - 1, Q <- Q (1 - D/2), contractions in
                         3xTF32 with FP32 accumulation (measured at chi = 130, d = 4:
                         max |B B^dag - 1| 9e-4 -> 1e-6 after 1xTF32; after 3xTF32 it is
                         already ~6e-7, the level the pass's Gram matrix resolves).
                         -1 (default): on for QRTEBD_C64_TF32 only; 0: off; 1: on. */
  int sweeps;         /* sweeps of the alternating least-squares solver that steps (i)-(ii)
                         are one of (Sec. II, comments after the algorithm): 0 or 1 (default)
                         is the paper's single sweep, enough for gates close to the identity;
                         k > 1 repeats X = theta~ Q^[n]^dag, QR, Y = Q^dag theta~, LQ with the
                         previous sweep's Q^[n] as Y0, for gates far from the identity (Sec. V:
                         circuit gates). eps never grows from sweep to sweep and reaches the
                         SVD optimum when the spectrum has a gap at eta. 1 <= k <= 1000. */
} qrtebd_trunc;
/* eta policy (Sec. II last paragraph, Sec. III):
 *   PLAIN: eta = min(chi_max, d chi_l, d chi_r); initial guess Y0 = B^n if
 *          eta == chi_m, else the first eta rows of theta~.
 *   CBE:   eta = min(chi_m + dchi, d chi_l, d chi_r); Y0 = first eta rows of theta~. */

/* Fill *tr with the defaults above for the given scheme and chi_max. */
int qrtebd_trunc_default(qrtebd_trunc* tr, int scheme, int chi_max);

/* ------------------------------------------------------------- bond update */
/* Inputs and outputs of one two-site update on the bond between sites m and
 * n = m + 1 (Fig. 2b / Fig. 3). All tensor pointers are DEVICE pointers in the
 * precision's storage type (complex128 for C128, complex64 otherwise), except
 * `gate`, which is always a device complex128 d^2 x d^2 matrix. */
typedef struct qrtebd_bond_io {
  int precision;             /* QRTEBD_C128 / C64_3XTF32 / C64_TF32 / C64_FP32 */
  int chi_l, d, chi_m, chi_r;
  int xi_kind;               /* 0: Xi = identity (xi unused); 1: dense chi_l x chi_l;
                                2: diagonal, xi holds chi_l complex entries;
                                3: dense chi_l x chi_l and lower triangular, its zeros stored
                                (the Xi~ = L / ||L|| a plain update writes): the product
                                Xi theta~' skips whole blocks above the diagonal, so entries
                                there must be zero */
  const void* xi;            /* Xi^[m] on the bond left of site m */
  const void* bm;            /* B^[m] (chi_l, d, chi_m); unused when theta != NULL */
  const void* bn;            /* B^[n] (chi_m, d, chi_r); right isometry */
  const void* theta;         /* optional theta' = B^m B^n (chi_l, d, d, chi_r): step (i)'s
                                contraction is then skipped and bm is not read */
  const void* gate;          /* U, device complex128 d^2 x d^2 */
  void* bm_out;              /* B~^[m] (chi_l, d, chi_new); capacity chi_l*d*eta */
  void* xi_out;              /* Xi~^[n] (chi_new, chi_new), ||Xi~||_F = 1; capacity eta*eta */
  void* bn_out;              /* B~^[n] (chi_new, d, chi_r); capacity eta*d*chi_r */
  double* stats_out;         /* optional device double[4]: eps, ||theta~||^2, kept norm^2,
                                chi_new. eps = ||theta~ - approx||^2 / ||theta~||^2 */
  double* schmidt_out;       /* optional device double[eta]: CBE Schmidt values S (descending,
                                unnormalised, all eta of them); ignored for PLAIN */
  void* workspace;           /* device scratch of at least qrtebd_bond_workspace_size bytes */
  size_t workspace_bytes;
} qrtebd_bond_io;

typedef struct qrtebd_bond_info {
  int eta;     /* expansion dimension used */
  int chi_new; /* new bond dimension chi~ (= eta for PLAIN) */
} qrtebd_bond_info;

/* Bytes of device workspace qrtebd_bond_update needs for these sizes (host call,
 * no GPU work). `xi_kind` as in qrtebd_bond_io; `theta_given` != 0 when the
 * caller supplies theta'. */
int qrtebd_bond_workspace_size(int precision, int chi_l, int d, int chi_m, int chi_r,
                               int xi_kind, int theta_given, const qrtebd_trunc* tr,
                               size_t* bytes);

/* One QR-TEBD bond update (Sec. II steps (i)-(iii); Sec. III steps (i)-(v) for CBE):
 *   theta' = B^m B^n (unless given); theta~' = U theta'; theta~ = Xi theta~';
 *   X = theta~ Y0^dag; Q R = X (Householder); Y = Q^dag theta~; L Q^[n] = Y (LQ);
 *   PLAIN: Xi~ = L / ||L||, B~^n = Q^[n];
 *   CBE:   L^dag L = V^dag S^2 V, keep chi~ values, B~^n = P V Q^[n], Xi~ = P S P / ||.||;
 *   B~^m = theta~' B~^n^dag (Hastings form, Sec. II).
 * Enqueued on `stream`. For PLAIN the call returns without synchronising; for
 * CBE every kernel after the cut reads chi~ on the device, and the call synchronises
 * `stream` once, after enqueuing all its work, to return chi~ in *info. Errors: INVALID_ARG for bad
 * sizes or eta > min(d chi_l, d chi_r) or eta > chi_m*... (see trunc), OOM if the
 * workspace is too small, CUDA on a launch failure, TIMEOUT if a kernel gave up a
 * bounded wait (reported at the next synchronising call). */
int qrtebd_bond_update(const qrtebd_bond_io* io, const qrtebd_trunc* tr, void* stream,
                       qrtebd_bond_info* info);

/* ------------------------------------------ CBE with Z_d charge sectors (Sec. III, last part)
 * With a global Z_d symmetry (for the clock model, Eqs. 2-3, the product of X over all sites,
 * in the basis where X is diagonal) every bond index carries a charge in 0..d-1 and the
 * tensors are block-sparse: B^i_{alpha beta} != 0 only if c(alpha) + i = c(beta) (mod d).
 * CBE expands every block of the central bond on its own and one cut over the Schmidt
 * values of all blocks picks chi~ and with it each block's dimension chi~_q, so the block
 * dimensions follow the state instead of being fixed before the step (Sec. III).
 *
 * Block q of theta~ (a (chi_l d) x (d chi_r) matrix, rows alpha*d + i, columns j*chi_r + delta)
 * holds the rows with c_l(alpha) + i = q and the columns with c_r(delta) - j = q, each in that
 * dense order. Per block: eta_q = min(chi_q + dchi_q, rows_q, cols_q), chi_q = the number of
 * old middle-bond states of charge q, dchi_q = max(tr->dchi_min, ceil(tr->dchi_frac chi_q));
 * Y0_q = the first eta_q rows of theta~_q; steps (i)-(iv) as in qrtebd_bond_update. The cut:
 * all Schmidt values in one descending list (equal values ordered by charge, then position),
 * then the rule of qrtebd_trunc (svd_min relative to the norm of all of them, chi_max,
 * eps_target, never inside a multiplet). The new middle bond lists the kept states block by
 * block in increasing charge, each block in descending Schmidt order. eps = 1 - kept /
 * ||theta~||^2 over all blocks (tr->eps_explicit is ignored). */
typedef struct qrtebd_sym_bond_io {
  int precision;           /* any QRTEBD_C* precision */
  int chi_l, d, chi_m, chi_r; /* 2 <= d <= 16 */
  const int* charge_l;     /* HOST int[chi_l]: charges of the left bond, 0..d-1 */
  const int* charge_m;     /* HOST int[chi_m]: charges of the old middle bond (sets chi_q) */
  const int* charge_r;     /* HOST int[chi_r]: charges of the right bond */
  int xi_kind;             /* 0: Xi = identity; 2: diagonal, xi holds chi_l entries */
  const void* xi;
  const void* theta;       /* theta' (chi_l, d, d, chi_r), device, storage type; only the
                              entries with c_l(alpha) + i + j = c_r(delta) are read */
  const void* bm;          /* with theta NULL: B^m (chi_l, d, chi_m) and B^n (chi_m, d, chi_r), */
  const void* bn;          /* device, and theta' = B^m B^n is formed first (one dense product) */
  const void* gate;        /* U, device complex128 d^2 x d^2, keeping i + j (mod d): only its
                              entries with i + j = i' + j' are read */
  void* bm_out;            /* B~^m (chi_l, d, chi_new), zero outside the charge rule;
                              capacity chi_l*d*cap, cap = min(chi_max, eta_sum) */
  void* xi_out;            /* the diagonal of Xi~ (chi_new entries, storage type, unit norm) */
  void* bn_out;            /* B~^n (chi_new, d, chi_r); capacity cap*d*chi_r */
  int* charge_out;         /* HOST int[cap]: charges of the new middle bond */
  int* chi_sector_out;     /* optional HOST int[d]: chi~_q */
  double* stats_out;       /* optional device double[4]: eps, ||theta~||^2, kept, chi_new */
  void* workspace;         /* device scratch of qrtebd_sym_bond_workspace_size bytes */
  size_t workspace_bytes;
} qrtebd_sym_bond_io;

/* Workspace bytes and eta_sum = sum_q eta_q for these charges (host call, no GPU work).
 * Errors: INVALID_ARG for d outside 2..16, a charge outside 0..d-1, a scheme other than
 * CBE, tr->eta != 0 or xi_kind 1 or 3. */
int qrtebd_sym_bond_workspace_size(int precision, int chi_l, int d, int chi_m, int chi_r,
                                   const int* charge_l, const int* charge_m, const int* charge_r,
                                   int xi_kind, int theta_given, const qrtebd_trunc* tr,
                                   size_t* bytes, int* eta_sum);

/* One charge-conserving CBE update, enqueued on `stream`: theta~'_q = U theta' gathered block
 * by block (one kernel), the blocks' dense CBE updates one after another, one cut over all
 * blocks and the scatter into the dense outputs on the device; the call synchronises `stream`
 * once at the end to fill charge_out / chi_sector_out and info (eta = eta_sum, chi_new).
 * Errors as qrtebd_bond_update. */
int qrtebd_sym_bond_update(const qrtebd_sym_bond_io* io, const qrtebd_trunc* tr, void* stream,
                           qrtebd_bond_info* info);

/* Synchronise `stream` and report any device-side error word (TIMEOUT / NUMERIC)
 * set by kernels since the last check. */
int qrtebd_stream_check(void* stream);

/* Failure detection (the paper has no counterpart). Every wait of a kernel on another
 * CTA is bounded; on expiry the kernel sets the device error word and returns, and the
 * next qrtebd_stream_check reports QRTEBD_ERR_TIMEOUT, leaving the context usable.
 * qrtebd_set_spin_limit: poll limit of the grid-wide barriers (the fused QR updates, the
 * CBE Jacobi sweeps) on the current device; polls <= 0 restores the default 2^24. The
 * mbarrier waits of the tensor-core and QR-panel pipelines keep the fixed 2^24 limit, as
 * their expiry path must drain copies still in flight. Synchronous host call.
 * qrtebd_selftest_barrier_timeout: enqueues on `stream` one CTA that waits at a grid
 * barrier sized for two CTAs, which nothing releases, so its bounded wait runs out; the
 * next qrtebd_stream_check on that stream then returns QRTEBD_ERR_TIMEOUT. */
int qrtebd_set_spin_limit(long long polls);
int qrtebd_selftest_barrier_timeout(void* stream);

/* ------------------------------------------------------------------ MPS state */
/* A matrix-product state in the right-isometric form of Sec. II (Eq. 1, Fig. 1):
 * site tensors B[m] (chi_m, d, chi_{m+1}) and bond matrices Xi[m] on the bond left
 * of site m, all resident in library-owned device memory.
 *   finite (infinite = 0): L sites, bonds 0..L, Xi[0] = Xi[L] = [[1]]; the gate on
 *     bond (m, m+1) reads Xi[m] and writes Xi[m+1] (Sec. II, finite systems).
 *   uniform (infinite = 1): unit cell of L sites (L even, >= 2), bonds 0..L-1 with
 *     wrap-around; the gate on (m, m+1 mod L) reads Xi[m], writes Xi[m+1 mod L].
 * Layers (Fig. 2a): parity 0 acts on the bonds (m, m+1) with m even, parity 1 on
 * m odd. A handle is bound to one stream and one device; it is not thread-safe. */
typedef struct qrtebd_mps qrtebd_mps;

typedef struct qrtebd_mps_desc {
  int L;                        /* sites (finite) or unit-cell length (uniform) */
  int d;                        /* local dimension, 2 <= d <= 8 */
  int infinite;                 /* 0 finite open chain, 1 uniform MPS */
  int chi_max;                  /* largest bond dimension the state may reach */
  int precision;                /* QRTEBD_C128 / C64_* as for qrtebd_bond_update */
  const double* product_state;  /* host complex128 L x d amplitudes (normalised per site),
                                   or NULL for |0 ... 0> (the Z = 1 state of Sec. IV) */
} qrtebd_mps_desc;

/* Allocate the state (device memory sized for chi_max on every bond, plus one
 * bond-update workspace) and initialise the product state: chi = 1 everywhere,
 * Xi = [[1]]. stream: cudaStream_t the handle uses for all its work.
 * Errors: INVALID_ARG (bad sizes, NULL out), OOM (device allocation failed). */
int qrtebd_mps_create(const qrtebd_mps_desc* desc, void* stream, qrtebd_mps** out);
/* Free all device memory of the state (synchronises its stream). NULL is a no-op. */
int qrtebd_mps_destroy(qrtebd_mps* mps);
/* Apply the two-site gates of one layer with the QR update (Sec. II / Sec. III).
 * gates_host: host complex128 array of nbonds x d^4 values, gate b acting on
 * (b, b+1) in the qrtebd.h gate layout; nbonds = L-1 (finite) or L (uniform); only
 * the bonds of `parity` are read and copied. tr: truncation for every bond.
 * eps_out: optional host array of nbonds doubles receiving each updated bond's eps
 * (others untouched); passing it synchronises the stream. Bonds of one layer are
 * independent (Fig. 2a): a layer of one bond is updated on the handle's stream; a layer
 * of two or more bonds runs on the worker-stream executor of
 * qrtebd_apply_gate_layer_batched (ordered after earlier work on the handle's stream and
 * before later work on it). */
int qrtebd_apply_gate_layer(qrtebd_mps* mps, int parity, const double* gates_host,
                            const qrtebd_trunc* tr, double* eps_out);
/* <O> at `site` (nsites = 1: op is d x d, Fig. 1c: tr[(Xi B)^dag O (Xi B)]) or on
 * (site, site+1) (nsites = 2: op is d^2 x d^2 in the gate layout, evaluated on
 * theta = Xi B^m B^n). op_host: host complex128. out: host double[2] (re, im).
 * Synchronises the stream. Accumulation in FP64. */
int qrtebd_expectation(qrtebd_mps* mps, int site, int nsites, const double* op_host,
                       double* out);
/* Truncation error eps accumulated on `bond` (the bond between sites bond-1 and
 * bond; for a uniform cell, index mod L) since creation, or summed over all bonds
 * when bond = -1. Synchronises. */
int qrtebd_truncation_error(qrtebd_mps* mps, int bond, double* out);
/* Schmidt values of bond `bond` (singular values of Xi, descending, normalised
 * to unit 2-norm) into host S (capacity entries); *n receives the bond dimension.
 * Synchronises. INVALID_ARG if capacity is too small. */
int qrtebd_schmidt(qrtebd_mps* mps, int bond, double* S, int capacity, int* n);
/* Von Neumann entanglement entropy of bond `bond` (Fig. 4 plots it on the central bond):
 * S_vN = -sum_k p_k ln p_k with p_k = S_k^2 from the normalised Schmidt values of
 * qrtebd_schmidt, natural log, FP64; terms with p_k <= 1e-300 are skipped. *out: host
 * double. Synchronises. INVALID_ARG for a bond outside the state or a NULL pointer. */
int qrtebd_entropy(qrtebd_mps* mps, int bond, double* out);
/* Current bond dimensions (finite: L+1 values, uniform: L values) into dims. */
int qrtebd_bond_dims(qrtebd_mps* mps, int* dims, int capacity, int* n);
/* Wait for all work on the handle's stream; reports device-side errors. */
int qrtebd_sync(qrtebd_mps* mps);
/* Checkpoint: write / read the whole state (tensors, bond dimensions, accumulated
 * eps) as a raw host dump. Loading with the same kernels reproduces the run bit
 * for bit. */
int qrtebd_mps_save(qrtebd_mps* mps, const char* path);
int qrtebd_mps_load(const char* path, void* stream, qrtebd_mps** out);

/* One layer (parity) applied to several states at once (the bonds of a layer are
 * independent, Fig. 2a). Every bond of `parity` of every state runs concurrently on a
 * pool of library-owned worker streams (one bond-update workspace each), ordered after
 * earlier work on each state's stream and before later work on it. gates_host[i]: the
 * gates of state i (as for qrtebd_apply_gate_layer); eps_out: NULL, or per-state arrays
 * (entries may be NULL) that receive each updated bond's eps (synchronises). For the
 * PLAIN scheme no host synchronisation happens; CBE keeps every cut on the device until the
 * whole layer is enqueued and then reads the new bond dimensions back once per state. A
 * layer whose shapes repeat (plain, or complex64 CBE) is recorded as a CUDA graph the second
 * time and replayed afterwards. A state may appear at most once. Not thread-safe per device. */
int qrtebd_apply_gate_layer_batched(qrtebd_mps* const* states, int nstates, int parity,
                                    const double* const* gates_host, const qrtebd_trunc* tr,
                                    double* const* eps_out);

/* Number of worker streams of the batched-layer executor. Each worker holds one bond-update
 * workspace sized for the largest bond it has run. Bonds whose workspace exceeds
 * QRTEBD_LAYER_BIG_BOND_BYTES run on the first QRTEBD_LAYER_BIG_WORKERS workers only (the
 * other bonds of such a layer on the rest), so a caller budgeting device memory for batched
 * layers (e.g. an admission policy) reserves QRTEBD_LAYER_BIG_WORKERS of its largest
 * workspaces plus, for the rest, workspaces of at most QRTEBD_LAYER_BIG_BOND_BYTES. */
#define QRTEBD_LAYER_BIG_BOND_BYTES (1024ull << 20)
#define QRTEBD_LAYER_BIG_WORKERS 8
int qrtebd_layer_workers(void);
/* Load a site tensor / bond matrix from host complex128 data (e.g. a random
 * right-canonical state, or a state produced elsewhere). B_host: (chi_l, d, chi_r);
 * sets the bond dimensions of bonds `site` and `site+1`. xi_host: chi x chi dense, or
 * chi diagonal entries when diagonal != 0. INVALID_ARG if a dimension exceeds the
 * state's capacity. Synchronises. The caller keeps neighbouring dimensions consistent. */
int qrtebd_mps_set_site(qrtebd_mps* mps, int site, const double* B_host, int chi_l, int chi_r);
int qrtebd_mps_set_bond(qrtebd_mps* mps, int bond, const double* xi_host, int chi, int diagonal);

/* -------------------------------------------------------------- complex GEMM */
/* C = alpha opA opB + beta C on device pointers, the contraction every step of
 * Sec. II is built from. opA(i, k) = A[i*sam + k*sak] (conjugated if conj_a),
 * opB(k, j) = B[k*sbk + j*sbn] (conjugated if conj_b), C(i, j) = C[i*scm + j*scn];
 * strides in complex elements, so transposes are stride choices. alpha, beta:
 * host complex128 (2 doubles each). precision as above: C128 / C64_FP32 run on
 * CUDA cores; C64_3XTF32 / C64_TF32 / C128_OZ on tcgen05 tensor cores and need
 * `workspace` of qrtebd_zgemm_workspace_size(m, n, k) bytes (device; NULL/0 allowed
 * for the CUDA-core precisions). C128_OZ runs products too small to fill the GPU on
 * the FP64 CUDA cores. Enqueued on `stream`, no synchronisation. */
int qrtebd_zgemm(int precision, int m, int n, int k, const void* A, long long sam, long long sak,
                 int conj_a, const void* B, long long sbk, long long sbn, int conj_b, void* C,
                 long long scm, long long scn, const double* alpha, const double* beta,
                 void* workspace, size_t workspace_bytes, void* stream);
size_t qrtebd_zgemm_workspace_size(int m, int n, int k);  /* enough for every precision */

/* Variant of qrtebd_zgemm that allocates nothing (the paper has no counterpart).
 * For callers that cannot call cudaMalloc around a GEMM: code recorded into a CUDA
 * graph under a capture mode that forbids allocation, latency-critical loops that
 * cannot afford an allocation or the device-wide synchronisation of a later free,
 * and frameworks that own all device memory through their own pool. The scratch
 * this GEMM needs (split/embedded TF32 operands, split-K partial sums) lives in one
 * file-scope device array of QRTEBD_NOALLOC_SCRATCH_BYTES, held on every GPU that
 * loads the library until the process exits; the caller still passes A, B and C.
 * precision: QRTEBD_C64_3XTF32 or QRTEBD_C64_TF32 only; m, n, k each at most
 * QRTEBD_NOALLOC_MAX_DIM, otherwise QRTEBD_ERR_INVALID_ARG with a message. Empty sizes
 * behave as in qrtebd_zgemm: m or n = 0 returns OK with nothing written, k = 0 scales C
 * by beta. Its kernels' waits are bounded: an expired wait returns nothing here, it sets
 * the device error word, which the next qrtebd_stream_check on `stream` reports as
 * QRTEBD_ERR_TIMEOUT. The first
 * call on a device looks up the array's device address (cudaGetSymbolAddress), so
 * make one call on each device before any stream capture. All calls share the array:
 * calls that overlap on the GPU (several streams or host threads) race on it and must
 * be serialised by the caller. Other arguments and semantics as qrtebd_zgemm. */
#define QRTEBD_NOALLOC_MAX_DIM 512
#define QRTEBD_NOALLOC_SCRATCH_BYTES 16777216
int qrtebd_zgemm_noalloc(int precision, int m, int n, int k, const void* A, long long sam,
                         long long sak, int conj_a, const void* B, long long sbk, long long sbn,
                         int conj_b, void* C, long long scm, long long scn, const double* alpha,
                         const double* beta, void* stream);

/* ------------------------------------------------------------ CBE decomposition */
/* Step (iv) of Sec. III on its own: for Rz (n x n device matrix, row-major, leading
 * dimension ldr, the precision's storage type), w (device double[n]) receives the
 * eigenvalues of Rz Rz^dag = L^dag L (L = Rz^dag; the squared singular values of L) in
 * descending order, and Vh (device complex128 n x n, row-major) the conjugated
 * eigenvectors as rows: Rz Rz^dag = Vh^dag diag(w) Vh. Complex64 precisions: one-sided
 * Jacobi in FP32 on the rows of Rz (FP64 norms and rotation parameters), one cooperative
 * launch; C128 / C128_OZ: the same one-sided Jacobi with FP64 rows, sums and rotations (one
 * cooperative launch) for n up to ~6800 (a pair of row blocks fits shared memory), beyond
 * that Rz Rz^dag in FP64 and a two-sided FP64 Jacobi. sweeps (device int, may be NULL):
 * Jacobi sweeps run by a one-sided solver (41 = stopped unconverged; 0 for the two-sided).
 * workspace: device, at least qrtebd_cbe_decompose_workspace_size bytes, else OOM.
 * INVALID_ARG for n < 1, ldr < n or a null pointer. Enqueued on `stream`. */
size_t qrtebd_cbe_decompose_workspace_size(int precision, int n);
int qrtebd_cbe_decompose(int precision, int n, const void* Rz, long long ldr, double* w, void* Vh,
                         void* workspace, size_t workspace_bytes, int* sweeps, void* stream);

/* ------------------------------------------------------------------ autotuner */
/* Tile shapes of the complex64 tensor-core products (batching pattern (2)). Every
 * product C = A B is run as a real GEMM over 128-row tiles of BN real output columns;
 * its launch configuration is (bn, splits, tail): bn = 128 or 256, splits = K-splits of
 * the whole grid (1 = none, 0 = the built-in heuristic), tail = with splits 1, whether a
 * short last wave of tiles runs with its K split over the idle SMs. A process-wide table
 * maps a product's shape (M, N, K, three = 3xTF32; after the library's N > M swap, so
 * M >= N) to the configuration measured fastest; shapes not in it use the heuristic.
 *
 * qrtebd_autotune_bond: runs one bond update of this shape on synthetic data on `stream`
 * (synchronously; not during stream capture), records the shapes of its tensor-core
 * products, then times every candidate configuration of each shape not yet in the table
 * on scratch operands (CUDA events, 2 warm-up + 5 timed runs) and stores the fastest.
 * Allocates its own device memory (cudaMalloc / cudaFree). Arguments as
 * qrtebd_bond_workspace_size; *n_shapes (may be NULL) receives the number of shapes
 * newly tuned. Precisions other than C64_3XTF32 / C64_TF32 tune nothing (OK).
 * qrtebd_autotune_entry: entry i in shape order: shape {M, N, K, three}, config
 * {bn, splits, tail}, ms {tuned, heuristic} (0 for entries set by hand).
 * qrtebd_autotune_set: insert or replace an entry (e.g. a table saved earlier).
 * The table is shared by all threads (a mutex guards it). */
int qrtebd_autotune_bond(int precision, int chi_l, int d, int chi_m, int chi_r, int xi_kind,
                         int theta_given, const qrtebd_trunc* tr, void* stream, int* n_shapes);
int qrtebd_autotune_count(void);
int qrtebd_autotune_entry(int i, int shape[4], int config[3], double ms[2]);
int qrtebd_autotune_set(const int shape[4], const int config[3]);
void qrtebd_autotune_clear(void);

/* Where the complex64 tensor-core products prepare their operands (the TF32 hi/lo split
 * and the 2 x 2 real embedding of B). Mode 1 (the default): a separate pass writes the
 * prepared operands to the workspace, and the GEMM loads them with TMA. Mode 0: inside
 * the GEMM kernel, whose epilogue warps convert the raw complex64 operands into its
 * shared-memory stages; this applies to products run with 128-column tiles whose operands
 * are contiguous along K or along their other index, with 16-byte aligned pairs. Other
 * products keep the separate pass. Other values: INVALID_ARG. The previous mode is
 * returned through *previous (may be NULL). The mode is process-wide. The two modes give
 * identical results: the same products, summed in the same order. The paper has no
 * counterpart to this tuning and diagnostic switch. */
int qrtebd_tc_operand_prep(int mode, int* previous);

/* ------------------------------------------------------------- Householder QR */
/* A = Q R for a device matrix A (m x n, m >= n, row-major, leading dimension lda, in the
 * precision's storage type): the factorisation of Sec. II (i) (and, applied to Y^dag,
 * the LQ of step (ii)). On return A holds R in its upper n x n triangle (real
 * diagonal, LAPACK geqrf sign convention) and zeros below; Q (m x n, ldq) holds the
 * explicit isometry. Blocked Householder: thread-block-cluster panels with FP64
 * reflector norms, compact-WY trailing updates. workspace: device, at least
 * qrtebd_qr_workspace_size bytes. Enqueued on `stream`; with more than two 128-column
 * blocks part of the work runs on two library-owned streams (a greatest-priority one for
 * the panel chain, a least-priority one for the look-ahead) forked from `stream` by events
 * and joined back into it, which stream capture records as graph edges. INVALID_ARG if
 * m < n, n < 1 or the panel does not fit shared memory. */
int qrtebd_householder_qr(int precision, int m, int n, void* A, long long lda, void* Q,
                          long long ldq, void* workspace, size_t workspace_bytes, void* stream);
size_t qrtebd_qr_workspace_size(int precision, int m, int n);

/* ------------------------------------------------------------- clock model */
/* Host-only: the clock-model bond gate U = exp(-i tau h_b) (Sec. IV, Eqs. 2-3) with
 * h_b = -(Z x Z^dag + Z^dag x Z) - g (wl (X + X^dag) x 1 + wr 1 x (X + X^dag)),
 * tau = tau_re + i tau_im. U_out: host complex128 d^2 x d^2. wl = wr = 1/2 except
 * at the outer site of a finite chain's end bonds (wl or wr = 1). */
int qrtebd_clock_bond_gate(int d, double g, double wl, double wr, double tau_re, double tau_im,
                           double* U_out);

/* Host-only: the same gate in the charge basis of the Z_d symmetry, (F x F)^dag U (F x F) with
 * F[n][k] = w^(nk) / sqrt(d) (column k: the eigenvector of X with eigenvalue w^k, so Z raises
 * the charge k by one); the entries with i + j != i' + j' (mod d), rounding noise of the basis
 * change, are set to zero. */
int qrtebd_clock_bond_gate_charge(int d, double g, double wl, double wr, double tau_re,
                                  double tau_im, double* U_out);

/* ------------------------------------------------------------ instrumentation */
/* Kernel families timed by qrtebd_profile_read. */
#define QRTEBD_PROF_TC_GEMM 0   /* tcgen05 complex GEMM kernel */
#define QRTEBD_PROF_QR_PANEL 1  /* cluster Householder panel kernel */
#define QRTEBD_PROF_SIMT_GEMM 2 /* CUDA-core complex GEMM kernel */
#define QRTEBD_PROF_PREP 3      /* tensor-core operand preparation (split / embed) */
#define QRTEBD_PROF_GATE 4      /* two-site gate application */
#define QRTEBD_PROF_BOND_GEMM 5 /* the bond-level contractions X = theta~ Y0^dag, Z = theta~^dag Q and
                                   the outputs (tensor-core or CUDA-core GEMM); the QR's
                                   own GEMMs count under QRTEBD_PROF_TC_GEMM / _SIMT_GEMM */
/* Number of kernels the library has launched since it was loaded (host counter). */
long long qrtebd_launch_count(void);
/* on != 0: record a CUDA event pair around every launch of the families above, on
 * the launching stream, from now on (earlier records are discarded); on == 0: stop. */
int qrtebd_profile_enable(int on);
/* Synchronise the recorded events of `family` and report their summed duration
 * (ms), number of launches, algorithmic flops and algorithmic bytes (any output
 * pointer may be NULL). */
int qrtebd_profile_read(int family, double* total_ms, long long* launches, double* flops,
                        double* bytes);

/* --------------------------------------------------------------- utilities */
const char* qrtebd_strerror(int status);
const char* qrtebd_last_error_message(void);
/* Library version string. */
const char* qrtebd_version(void);

#ifdef __cplusplus
}
#endif

#endif /* QRTEBD_H */
