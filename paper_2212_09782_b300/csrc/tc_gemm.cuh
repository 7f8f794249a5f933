// Complex64 GEMM on sm_103a tensor cores (tcgen05, kind::tf32, TMEM accumulators).
//
// A complex product C = opA * opB becomes one real GEMM C' = A' B'^T:
//   A' (M x 2K): row m = (Re, Im) of opA(m, k) interleaved - the natural
//                complex64 layout of a K-contiguous operand;
//   B'^T (2N x 2K): rows 2n and 2n+1 hold (Re b, -Im b) and (Im b, Re b) for
//                b = opB(k, n) (the 2 x 2 real embedding of a complex number);
//   C' (M x 2N) is then C in the interleaved complex layout: 8 real flops per
//   complex multiply-add, no wasted work.
// 3xTF32: every operand is split x = hi + lo with hi = tf32(x), and the MMA
// pipe accumulates hi*hi + hi*lo + lo*hi in FP32 (about FP32 accuracy).
#pragma once
#include "common.cuh"
#include "gemm_simt.cuh"

#include <vector>

namespace qrtebd {

struct TcSlot {
  float* hi = nullptr;
  float* lo = nullptr;
  // cache key of the prepared operand (valid within one bond update)
  const void* src = nullptr; long long s0 = 0, s1 = 0; int rows = 0, cols = 0; bool conj = false;
  bool three = false; bool valid = false; int ld = 0;
};

struct TcWorkspace {
  TcSlot a[2];  // a[0]: an operand marked for reuse; a[1]: every other A'
  TcSlot b;
  size_t a_cap = 0, b_cap = 0;  // floats per hi (or lo) array
  float* partial = nullptr;     // split-K partial sums
  size_t p_cap = 0;             // floats
};

// Carve operand buffers able to hold A' for max_m x max_k and B'^T for max_n x max_k.
void tc_carve(Arena& ar, int max_m, int max_k, int max_n, TcWorkspace& w);

// Shapes worth (and able to be) run on the tensor cores.
bool tc_gemm_eligible(const GemmArgs<float>& g);

// C = alpha opA opB + beta C through tcgen05. Falls back to the CUDA-core GEMM
// when the prepared operands would not fit the workspace.
int tc_gemm(const GemmArgs<float>& g, bool three, TcWorkspace& w, cudaStream_t st,
            int prof_family = PROF_TC_GEMM);

// Invalidate cached prepared operands (call when their sources may change).
void tc_invalidate(TcWorkspace& w);

// ---- complex128 GEMM by FP64 emulation on the TF32 tensor cores (Ozaki splitting)
// Every row of A' (and of the embedded B'^T) is scaled by a power of two to |x| < 1 and cut
// into OZ_SLICES integer slices of OZ_BITS bits, x 2^-E = sum_p d_p 2^(-OZ_BITS (p+1)) with
// |d_p| <= 2^OZ_BITS, each exactly representable in TF32. A slice product summed over 1024 K
// terms stays within 2^24, so the tensor core's FP32 accumulation is exact; every such chunk
// is added into FP64 registers with its weight 2^(-OZ_BITS (p+q+2)), over the slice pairs
// p + q <= OZ_SLICES - 1 (0-based). Truncation error ~2^-56 of |A||B| per K term, below the
// complex128 rounding of the result.
constexpr int OZ_SLICES = 8;
constexpr int OZ_BITS = 7;
struct OzWorkspace {
  unsigned short* a = nullptr;  // FP16 slices: OZ_SLICES x max_m rows x ld halves
  unsigned short* b = nullptr;  // OZ_SLICES x 2 max_n rows x ld halves
  int* ea = nullptr;   // per row of A' (max_m)
  int* eb = nullptr;   // per complex column of opB (max_n)
  double2* part = nullptr;  // partial tiles of a product whose slice pairs are split over CTAs
  size_t a_cap = 0, b_cap = 0, ea_cap = 0, eb_cap = 0, part_cap = 0;
};
void oz_carve(Arena& ar, int max_m, int max_k, int max_n, OzWorkspace& w);
// Shapes worth (and able to be) run on the tensor cores in emulated FP64.
bool oz_gemm_eligible(const GemmArgs<double>& g);
// C = alpha opA opB + beta C (complex128) on the tensor cores; falls back to the FP64
// CUDA-core GEMM when the slices would not fit the workspace.
int oz_gemm(const GemmArgs<double>& g, OzWorkspace& w, cudaStream_t st, int prof_family = PROF_TC_GEMM);

// ---- launch configurations and the autotuner's table
// A product's shape as the kernel sees it (after the N > M swap): M >= N.
struct TcShape {
  int M, N, K, three;
  bool operator<(const TcShape& o) const {
    return M != o.M ? M < o.M : N != o.N ? N < o.N : K != o.K ? K < o.K : three < o.three;
  }
};
// bn: real output columns per tile (128 or 256); splits: K-splits of the whole grid
// (>= 1; 0 = the heuristic); tail: with splits == 1, whether a short last wave runs
// with its K split over the idle SMs.
struct TcConfig { int bn = 256; int splits = 0; int tail = 1; };
struct TcTuned { TcShape shape; TcConfig cfg; double ms_tuned, ms_default; };

// C = alpha opA opB + beta C with a given configuration (nullptr: the table's entry for
// the shape, else the heuristic).
int tc_gemm_cfg(const GemmArgs<float>& g, bool three, TcWorkspace& w, cudaStream_t st,
                const TcConfig* cfg, int prof_family = PROF_TC_GEMM);
// Shapes seen by tc_gemm between begin and end (the tuner's recording pass).
void tc_record_begin();
std::vector<TcShape> tc_record_end();
// Time the candidate configurations of one shape on scratch operands (synchronous, not
// during stream capture) and store the fastest in the table.
int tc_tune_shape(const TcShape& s, cudaStream_t st, TcTuned* out);
bool tc_tune_get(const TcShape& s, TcConfig* cfg);
void tc_tune_put(const TcTuned& t);
std::vector<TcTuned> tc_tune_list();
void tc_tune_clear();
// Operand preparation: 0 inside the GEMM kernel (where the layout allows), 1 separate pass.
int tc_prep_mode(int mode);  // sets the mode, returns the previous one

}  // namespace qrtebd
