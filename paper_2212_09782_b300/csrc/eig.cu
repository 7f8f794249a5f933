// Hermitian eigensolver for CBE step (iv) (Sec. III: diagonalise L^dag L = V^dag S^2 V).
//
// Parallel cyclic Jacobi in FP64 with the round-robin (circle) ordering: each
// of the n'-1 steps of a sweep (n' = n rounded up to even) rotates n'/2
// disjoint index pairs at once. A rotation G on (p, q), with a_pq = |a| e,
//   G = [[c, s e], [-s conj(e), c]],  t = tan(theta) = sign(z) / (|z| + sqrt(1 + z^2)),
//   z = (a_qq - a_pp) / (2 |a|),  c = 1 / sqrt(1 + t^2),  s = t c,
// zeroes (G^dag A G)_pq. Sweeps repeat until the off-diagonal Frobenius norm is
// below 1e-15 of the total (checked on the host once per sweep).
//
// For complex64 the solver of record is instead a one-sided Jacobi SVD in FP32 on the rows
// of Rz (svd_rows_jacobi32 below): L^dag L = Rz Rz^dag is never formed, the singular
// values come out with the relative accuracy of the FP32 input rather than squared, and
// the whole iteration is one cooperative launch.
#include "bond.cuh"

#include <algorithm>
#include <cmath>
#include <mutex>

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
  auto key = [](double x) { return isnan(x) ? -INFINITY : x; };  // ranks stay a permutation
  double li = key(A[(long long)i * n + i].x);
  int rank = 0;
  for (int j = 0; j < n; ++j) {
    double lj = key(A[(long long)j * n + j].x);
    if (lj > li || (lj == li && j < i)) ++rank;
  }
  w[rank] = A[(long long)i * n + i].x;
  for (int r = 0; r < n; ++r) {
    double2 v = V[(long long)r * n + i];
    Vh[(long long)rank * n + r] = make_double2(v.x, -v.y);
  }
}

// ------------------------------------------------------------ one-sided Jacobi (FP32)
// Rows r_i of R (n x n) are rotated in pairs until every pair is orthogonal to `tol`
// (|r_p r_q^dag| <= tol ||r_p|| ||r_q||), the same rotations applied to Jt (from 1): then
// Jt Rz = R has orthogonal rows, Rz Rz^dag = Jt^dag diag(||r_i||^2) Jt, and the rows of
// Jt are the conjugated eigenvectors of L^dag L = Rz Rz^dag (L = Rz^dag), ||r_i|| its
// singular values. A pair's rotation is the 2 x 2 Hermitian Jacobi step of the rows'
// Gram matrix [[a, g], [conj g, b]] (a = ||r_p||^2, b = ||r_q||^2, g = r_p r_q^dag), as in
// k_jac_rot: rows p, q <- G^dag (rows p, q).
// Blocked: the rows form blocks of br (4, 2 or 1, the largest whose block pair fits
// shared memory; the row count is padded with zero rows to a multiple of br). A sweep
// pairs the blocks in the round-robin order (nb'/2 disjoint block pairs per round, nb'-1
// rounds); one CTA per block pair loads its 2 br rows into shared memory, rotates its
// br^2 cross pairs (br inner rounds of br disjoint pairs), writes the rows back and applies
// the accumulated 2br x 2br rotation W to the same rows of Jt; the pairs inside a block
// get one such visit per sweep before the rounds. A grid barrier separates the rounds;
// sweeps repeat until one applies no rotation (at most SJ_MAX_SWEEPS). No FP64
// instruction in the loop (B300's FP64 pipe, about one FMA per clock per SM, made the
// reductions alone the critical path): the rows are FP32, the partial sums of r_a r_b^dag
// are combined across the pair's warps in double-float (TwoSum), the rows' squared norms
// are summed the same way once per visit and then updated in closed form by each rotation,
// and the rotation is formed in FP32 from those sums with c = 1 - t^2/(q(1+q)),
// q = sqrt(1+t^2), rounded once. Both matter: an FP32 tree, or c = 1/q directly, each
// left the singular values ~10x less accurate (an FP32 emulation at n = 256: 1.4e-5 vs
// 1.1e-6 relative to the largest squared value). The rotations are unitary only to
// rounding, and ~10^4 of them per row drift its norm by ~1e-5; the same rotations act on R
// and Jt, so the outputs use the ratio: S_i^2 = ||r_i||^2 / ||j_i||^2 and the rows of Jt
// normalised (at n = 1126 this took the rows' orthonormality from 3e-5 to 3e-6 and
// sum_i S_i^2 to within 1e-7 of ||Rz||^2). Global loads bypass L1 (ld.global.cg): other
// CTAs rewrite rows between rounds.
constexpr int SJ_BRMAX = 4;                      // rows per block (8 and 2 measured slower)
constexpr int SJ_WPP = 2;                        // warps per row pair
constexpr int SJ_NT = 32 * SJ_WPP * SJ_BRMAX;    // 256: SJ_WPP warps for each of br pairs
constexpr int SJ_MAX_SWEEPS = 40;
struct SjCtl {
  unsigned bar[2];
  unsigned rot[SJ_MAX_SWEEPS];  // rotations applied per sweep
  int sweeps;                   // sweeps run; SJ_MAX_SWEEPS + 1: not converged
};

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// double-float (hi, lo) sums in FP32 arithmetic (TwoSum): the rows' Gram entries to ~FP64
// accuracy without FP64 instructions
struct DF { float hi, lo; };
__device__ __forceinline__ DF df_add(DF a, DF b) {
  const float s = a.hi + b.hi, v = s - a.hi;
  float e = (a.hi - (s - v)) + (b.hi - v);
  e += a.lo + b.lo;
  const float h = s + e;
  return DF{h, e - (h - s)};
}
// the lane's two partial sums, then the whole warp (every lane ends with the total)
__device__ __forceinline__ DF warp_sum_df2(const float f[2]) {
  DF v = df_add(DF{f[0], 0.f}, DF{f[1], 0.f});
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    v = df_add(v, DF{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)});
  return v;
}

__host__ __device__ inline size_t sj_smem_bytes(int n, int br) {
  return (size_t)2 * br * n * sizeof(float2) + (size_t)(2 * SJ_BRMAX) * (2 * SJ_BRMAX) * sizeof(float2);
}

// n: the row length (even; a zero column pads an odd order), nb: blocks of br rows.
// A sweep visits every row pair once: first each block alone (its br(br-1)/2 pairs, one
// CTA per block), then the block round robin, where a block pair's visit handles only its
// br x br cross pairs (br inner rounds pairing row i of the first block with row
// (i + j) mod br of the second). SJ_WPP warps share a row pair: each sums its share of the
// row, the pair's warps combine their partials through shared memory behind a named
// barrier, and each then forms the same rotation and applies it to its own share.
__global__ void __launch_bounds__(SJ_NT, 1) k_sj_sweeps(float2* R, float2* Jt, int n, int br, int nb,
                                                        double tol, SjCtl* ctl, unsigned* err) {
  extern __shared__ __align__(16) unsigned char sj_sm[];
  float2* X = reinterpret_cast<float2*>(sj_sm);              // [2 br][n]
  float2* Wm = X + (size_t)2 * br * n;                         // [2 br][2 br]
  __shared__ float red[SJ_BRMAX][SJ_WPP][4];                   // per pair slot and warp: g (hi, lo)
  __shared__ DF nrm[2 * SJ_BRMAX];                             // ||row||^2 of the rows held
  __shared__ unsigned s_cnt, s_vis;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int quad = warp / SJ_WPP, qw = warp % SJ_WPP;          // pair slot, warp within it
  const int qt = qw * 32 + lane;                               // thread within the pair slot
  const int nbp = (nb % 2) ? nb + 1 : nb;   // blocks, with an idle partner when odd
  const float tolf = (float)tol;

  // One visit: rows grow(0..nrow-1) into shared memory, the inner rounds (cross: br rounds
  // of br pairs between the halves; else the round robin among the nrow rows), then the
  // rows back and W applied to the same rows of Jt when anything rotated.
  auto visit = [&](int nrow, bool cross, auto grow) {
    {
      // 16-byte asynchronous copies that bypass L1, all in flight at once (n is even: rows
      // are 16-byte aligned)
      const int h = n / 2, tot = nrow * h;
      for (int idx = tid; idx < tot; idx += SJ_NT) {
        const int a = idx / h, o = 2 * (idx - a * h);
        const float2* src = R + (long long)grow(a) * n + o;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                         (unsigned)__cvta_generic_to_shared(X + (size_t)a * n + o)),
                     "l"(src)
                     : "memory");
      }
      asm volatile("cp.async.wait_all;" ::: "memory");
    }
    for (int e = tid; e < nrow * nrow; e += SJ_NT) Wm[e] = make_float2(e / nrow == e % nrow ? 1.f : 0.f, 0.f);
    if (tid == 0) s_vis = 0;
    __syncthreads();
    // the rows' squared norms once per visit (double-float); each rotation then updates them
    // in closed form, a' = a - t|g|, b' = b + t|g|, so the inner rounds sum only g
    for (int a = warp; a < nrow; a += SJ_NT / 32) {
      const float2* xr = X + (size_t)a * n;
      float f[2] = {0.f, 0.f};
      int i = lane;
      for (; i + 32 < n; i += 64) {
        const float2 x = xr[i], y = xr[i + 32];
        f[0] = fmaf(x.x, x.x, fmaf(x.y, x.y, f[0]));
        f[1] = fmaf(y.x, y.x, fmaf(y.y, y.y, f[1]));
      }
      if (i < n) { const float2 x = xr[i]; f[0] = fmaf(x.x, x.x, fmaf(x.y, x.y, f[0])); }
      const DF v = warp_sum_df2(f);
      if (lane == 0) nrm[a] = v;
    }
    __syncthreads();
    const int rounds = cross ? br : nrow - 1;
    const int pairs = cross ? br : nrow / 2;
    for (int ir = 0; ir < rounds; ++ir) {
      if (quad < pairs) {                   // slot-uniform
        int a, b;
        if (cross) { a = quad; b = br + (quad + ir) % br; }
        else pair_of(ir, quad, nrow, a, b);
        float2* xa = X + (size_t)a * n;
        float2* xb = X + (size_t)b * n;
        float fr[2] = {0, 0}, fi[2] = {0, 0};
        auto acc = [&](int u, int j) {
          const float2 x = xa[j], y = xb[j];
          fr[u] = fmaf(x.x, y.x, fmaf(x.y, y.y, fr[u]));   // Re(x conj y)
          fi[u] = fmaf(x.y, y.x, fmaf(-x.x, y.y, fi[u]));  // Im(x conj y)
        };
        constexpr int QT = 32 * SJ_WPP;
        int i = qt;
        for (; i + QT < n; i += 2 * QT) { acc(0, i); acc(1, i + QT); }
        if (i < n) acc(0, i);
        DF sums[2] = {warp_sum_df2(fr), warp_sum_df2(fi)};
        if (SJ_WPP > 1) {
          if (lane == 0) {
#pragma unroll
            for (int v = 0; v < 2; ++v) { red[quad][qw][2 * v] = sums[v].hi; red[quad][qw][2 * v + 1] = sums[v].lo; }
          }
          asm volatile("bar.sync %0, %1;" ::"r"(1 + quad), "n"(32 * SJ_WPP) : "memory");
#pragma unroll
          for (int v = 0; v < 2; ++v) {     // the slot's total, in the same order in every warp
            DF t{red[quad][0][2 * v], red[quad][0][2 * v + 1]};
#pragma unroll
            for (int w = 1; w < SJ_WPP; ++w) t = df_add(t, DF{red[quad][w][2 * v], red[quad][w][2 * v + 1]});
            sums[v] = t;
          }
        }
        const DF Ad = nrm[a], Bd = nrm[b];
        const float A = Ad.hi, B = Bd.hi, Gr = sums[0].hi, Gi = sums[1].hi;
        const float ab = hypotf(Gr, Gi);
        // |g| below 1e-30 is a product of rows at the FP32 noise floor of a unit-norm
        // matrix; the floor also keeps 1/|g| finite (a denormal |g| overflowed it)
        if (ab > 1e-30f && ab > tolf * sqrtf(A) * sqrtf(B)) {  // slot-uniform
          const float inv = 1.f / ab;
          // z = (b - a) / 2|g| with b - a from the double-float norms (no cancellation)
          const float z = ((Bd.hi - Ad.hi) + (Bd.lo - Ad.lo)) * (0.5f * inv);
          // t = tan(theta); for |z| beyond 1e18, 1 + z^2 overflows and t = 1/(2z) ~ 0
          const float t = fabsf(z) > 1e18f ? 0.5f / z
                                           : copysignf(1.f, z) / (fabsf(z) + sqrtf(fmaf(z, z, 1.f)));
          // c = 1/sqrt(1 + t^2) as 1 - t^2 / (q (1 + q)), q = sqrt(1 + t^2): rounded once,
          // so that small rotations do not drift the norms (c ~ 1 - t^2/2 rounded to 1)
          const float qq = sqrtf(fmaf(t, t, 1.f));
          const float c = 1.f - (t * t) / (qq * (1.f + qq)), sn = t * c;
          const float er = sn * (Gr * inv), ei = sn * (Gi * inv);
          // row_a' = c x - (s e) y ; row_b' = conj(s e) x + c y (each warp its share)
          for (int j2 = qt; j2 < n; j2 += QT) {
            const float2 x = xa[j2], y = xb[j2];
            xa[j2] = make_float2(c * x.x - (er * y.x - ei * y.y), c * x.y - (er * y.y + ei * y.x));
            xb[j2] = make_float2((er * x.x + ei * x.y) + c * y.x, (er * x.y - ei * x.x) + c * y.y);
          }
          if (qw == 0) {
            if (lane < nrow) {
              const float2 x = Wm[a * nrow + lane], y = Wm[b * nrow + lane];
              Wm[a * nrow + lane] = make_float2(c * x.x - (er * y.x - ei * y.y), c * x.y - (er * y.y + ei * y.x));
              Wm[b * nrow + lane] = make_float2((er * x.x + ei * x.y) + c * y.x, (er * x.y - ei * x.x) + c * y.y);
            }
            if (lane == 0) {
              atomicAdd(&s_vis, 1u);
              const float tg = t * ab, tge = fmaf(t, ab, -tg);  // t|g| exactly as hi + lo
              nrm[a] = df_add(Ad, DF{-tg, -tge});
              nrm[b] = df_add(Bd, DF{tg, tge});
            }
          }
        }
      }
      __syncthreads();  // the next inner round pairs other rows; red and nrm are reused
    }
    if (s_vis) {
      const int h = n / 2, tot = nrow * h;
      for (int idx = tid; idx < tot; idx += SJ_NT) {
        const int a = idx / h, o = 2 * (idx - a * h);
        *reinterpret_cast<float4*>(R + (long long)grow(a) * n + o) =
            *reinterpret_cast<const float4*>(X + (size_t)a * n + o);
      }
      for (int c = tid; c < n; c += SJ_NT) {
        float2 in[2 * SJ_BRMAX];
#pragma unroll
        for (int a = 0; a < 2 * SJ_BRMAX; ++a)
          if (a < nrow) in[a] = __ldcg(Jt + (long long)grow(a) * n + c);
#pragma unroll
        for (int a = 0; a < 2 * SJ_BRMAX; ++a) {
          if (a < nrow) {
            float2 o = make_float2(0.f, 0.f);
#pragma unroll
            for (int b = 0; b < 2 * SJ_BRMAX; ++b) {
              if (b < nrow) {
                const float2 wv = Wm[a * nrow + b];
                o.x = fmaf(wv.x, in[b].x, fmaf(-wv.y, in[b].y, o.x));
                o.y = fmaf(wv.x, in[b].y, fmaf(wv.y, in[b].x, o.y));
              }
            }
            Jt[(long long)grow(a) * n + c] = o;
          }
        }
      }
      if (tid == 0) s_cnt += s_vis;
    }
    __syncthreads();  // X, Wm and s_vis are reused by the next visit
  };

  for (int sweep = 0; sweep < SJ_MAX_SWEEPS; ++sweep) {
    if (tid == 0) s_cnt = 0;
    if (br > 1) {  // the pairs inside each block
      for (int blk = blockIdx.x; blk < nb; blk += gridDim.x)
        visit(br, false, [&](int a) { return blk * br + a; });
      if (!grid_barrier(ctl->bar, gridDim.x, err)) return;
    }
    for (int r = 0; r < nbp - 1; ++r) {  // the cross pairs of each block pair
      for (int k = blockIdx.x; k < nbp / 2; k += gridDim.x) {
        int P, Q;
        pair_of(r, k, nbp, P, Q);
        if (Q < nb)                          // uniform in the CTA; the idle partner has none
          visit(2 * br, true, [&](int a) { return a < br ? P * br + a : Q * br + (a - br); });
      }
      if (!grid_barrier(ctl->bar, gridDim.x, err)) return;
    }
    if (tid == 0 && s_cnt) atomicAdd(&ctl->rot[sweep], s_cnt);
    if (!grid_barrier(ctl->bar, gridDim.x, err)) return;
    if (*reinterpret_cast<volatile unsigned*>(&ctl->rot[sweep]) == 0) {
      if (blockIdx.x == 0 && tid == 0) ctl->sweeps = sweep + 1;
      return;
    }
  }
  if (blockIdx.x == 0 && tid == 0) ctl->sweeps = SJ_MAX_SWEEPS + 1;
}

__global__ void k_eye32(float2* J, int n, int ld) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)n * n) return;
  const long long r = idx / n, c = idx % n;
  J[r * ld + c] = make_float2(r == c ? 1.f : 0.f, 0.f);
}

// s2[i] = ||r_i||^2 / ||j_i||^2 and jn[i] = 1 / ||j_i|| in FP64, one warp per row. The FP32
// rotations are unitary only to rounding, and the same ones act on R and Jt, so the drift of
// a row's norm (~1e-5 after ~10^4 rotations) cancels in the ratio.
__global__ void k_sj_norms(const float2* R, const float2* Jt, int n, int ld, double* s2, double* jn) {
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (row >= n) return;
  double acc = 0.0, accj = 0.0;
  for (int i = lane; i < n; i += 32) {
    const float2 x = R[(long long)row * ld + i], y = Jt[(long long)row * ld + i];
    acc = fma((double)x.x, (double)x.x, fma((double)x.y, (double)x.y, acc));
    accj = fma((double)y.x, (double)y.x, fma((double)y.y, (double)y.y, accj));
  }
  acc = warp_sum_d(acc);
  accj = warp_sum_d(accj);
  if (lane == 0) {
    s2[row] = accj > 0 ? acc / accj : acc;
    jn[row] = accj > 0 ? 1.0 / sqrt(accj) : 1.0;
  }
}

// descending order of s2 (stable): w[rank] = s2[i], order[rank] = i. A NaN sorts as -inf,
// so the ranks are a permutation whatever the values (order[] is then fully written).
__global__ void k_sj_rank(const double* s2, int n, double* w, int* order) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  auto key = [](double x) { return isnan(x) ? -INFINITY : x; };
  const double li = key(s2[i]);
  int rank = 0;
  for (int j = 0; j < n; ++j) {
    const double lj = key(s2[j]);
    if (lj > li || (lj == li && j < i)) ++rank;
  }
  w[rank] = s2[i];
  order[rank] = i;
}

// Vh[rank] = row order[rank] of Jt, normalised (FP64); an index out of range (impossible
// while order is a permutation) sets DEVERR_BOUNDS and is skipped
__global__ void k_sj_gather(const float2* Jt, const int* order, const double* jn, int n, int ld,
                            double2* Vh, unsigned* err) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)n * n) return;
  const int r = (int)(idx / n), c = (int)(idx % n);
  const int src = order[r];
  if (src < 0 || src >= n) {
    if (c == 0) atomicOr(err, DEVERR_BOUNDS);
    return;
  }
  const float2 v = Jt[(long long)src * ld + c];
  const double f = jn[src];
  Vh[idx] = make_double2(f * v.x, f * v.y);
}

// rows per block: the largest of 8, 4, 2, 1 whose block pair fits the shared memory
int sj_rows_per_block(int n) {
  for (int br = SJ_BRMAX; br > 1; br /= 2)
    if (sj_smem_bytes(n, br) <= 200 * 1024) return br;
  return sj_smem_bytes(n, 1) <= 220 * 1024 ? 1 : 0;
}

int sj_grid(int npairs, size_t smem) {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sj_sweeps, SJ_NT, smem) != cudaSuccess)
    return 0;
  return std::min(npairs, std::min(sms * per, 2 * sms));
}

}  // namespace

size_t svd32_work_bytes(int n) {
  const int ld = n + (n & 1);
  const int br = std::max(1, sj_rows_per_block(ld));
  const size_t rows = (size_t)ceil_div(n, br) * br;  // padded with zero rows
  return align_up(2 * rows * ld * sizeof(float2), 256) + align_up((size_t)n * sizeof(double), 256) +
         align_up((size_t)n * sizeof(int), 256) + align_up(sizeof(SjCtl), 256) +
         align_up((size_t)n * sizeof(double), 256);
}

int svd_rows_jacobi32(const float2* Rz, long long ldr, int n, double* w, double2* Vh, void* work,
                      size_t work_bytes, cudaStream_t st, unsigned* err, int* sweeps) {
  if (n < 1 || ldr < n || !Rz || !w || !Vh || !work || work_bytes < svd32_work_bytes(n))
    return QRTEBD_ERR_INVALID_ARG;
  const int ld = n + (n & 1);  // even row length: 16-byte aligned rows
  const int br = sj_rows_per_block(ld);
  if (br < 1) { set_last_message("svd_rows_jacobi32: rows too long for shared memory"); return QRTEBD_ERR_INVALID_ARG; }
  const int nb = (int)ceil_div(n, br);
  const size_t rows = (size_t)nb * br;
  char* q = static_cast<char*>(work);
  float2* R = reinterpret_cast<float2*>(q);
  float2* Jt = R + rows * ld;
  q += align_up(2 * rows * ld * sizeof(float2), 256);
  double* s2 = reinterpret_cast<double*>(q); q += align_up((size_t)n * sizeof(double), 256);
  int* order = reinterpret_cast<int*>(q); q += align_up((size_t)n * sizeof(int), 256);
  SjCtl* ctl = reinterpret_cast<SjCtl*>(q); q += align_up(sizeof(SjCtl), 256);
  double* jn = reinterpret_cast<double*>(q);
  // R = Rz, Jt = identity; zero rows below and a zero column right of them when n is odd
  QR_CUDA_TRY(cudaMemsetAsync(R, 0, 2 * rows * ld * sizeof(float2), st));
  QR_CUDA_TRY(cudaMemcpy2DAsync(R, (size_t)ld * sizeof(float2), Rz, (size_t)ldr * sizeof(float2),
                                (size_t)n * sizeof(float2), (size_t)n, cudaMemcpyDeviceToDevice, st));
  k_eye32<<<(unsigned)ceil_div((long long)n * n, 256), 256, 0, st>>>(Jt, n, ld);
  note_launch();
  QR_CUDA_TRY(cudaGetLastError());
  QR_CUDA_TRY(cudaMemsetAsync(ctl, 0, sizeof(SjCtl), st));
  if (n > 1) {
    const size_t smem = sj_smem_bytes(ld, br);
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] {
      attr = cudaFuncSetAttribute(k_sj_sweeps, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    });
    QR_CUDA_TRY(attr);
    const int nbp = (nb % 2) ? nb + 1 : nb;
    const int grid = sj_grid(nbp / 2, smem);
    if (grid < 1) { set_last_message("svd_rows_jacobi32: no resident CTA"); return QRTEBD_ERR_CUDA; }
    // convergence: orthogonal to FP32 working accuracy, sqrt(n) eps (the rows' rounding)
    double tol = std::sqrt((double)std::max(n, 16)) * 5.96e-8;
    int nv = ld, brv = br, nbv = nb;
    void* args[] = {&R, &Jt, &nv, &brv, &nbv, &tol, &ctl, &err};
    QR_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_sj_sweeps, dim3((unsigned)grid), dim3(SJ_NT),
                                            args, smem, st));
    note_launch();
  }
  k_sj_norms<<<(unsigned)ceil_div(n, 8), 256, 0, st>>>(R, Jt, n, ld, s2, jn);
  note_launch();
  k_sj_rank<<<(unsigned)ceil_div(n, 128), 128, 0, st>>>(s2, n, w, order);
  note_launch();
  k_sj_gather<<<(unsigned)ceil_div((long long)n * n, 256), 256, 0, st>>>(Jt, order, jn, n, ld, Vh, err);
  note_launch();
  QR_CUDA_TRY(cudaGetLastError());
  if (sweeps) QR_CUDA_TRY(cudaMemcpyAsync(sweeps, &ctl->sweeps, sizeof(int), cudaMemcpyDeviceToDevice, st));
  return QRTEBD_OK;
}

namespace {

// ---------------------------------------------------------------- one-sided Jacobi, FP64
// The complex128 form of svd_rows_jacobi32: the same blocked one-sided Jacobi on the rows of
// Rz (block pairs in the round-robin order, one CTA per block pair, a bounded grid barrier
// between rounds, the whole iteration one cooperative launch), with the rows, the Gram sums
// and the rotations in FP64. It replaces the two-sided solver for CBE step (iv) in
// complex128: that one issues three launches per rotation step and reads the off-diagonal
// norm back once per sweep (~10^4 launches and ~10 stream synchronisations at n ~ 300).
// The singular values of L come out with the relative accuracy of the FP64 rows, and
// L^dag L is never formed.
constexpr int SJ64_BRMAX = 4;
constexpr int SJ64_WPP = 2;
constexpr int SJ64_NT = 32 * SJ64_WPP * SJ64_BRMAX;  // 256
constexpr int SJ64_MAX_SWEEPS = 40;
struct Sj64Ctl {
  unsigned bar[2];
  unsigned rot[SJ64_MAX_SWEEPS];
  int sweeps;
};

__host__ __device__ inline size_t sj64_smem_bytes(int n, int br) {
  return (size_t)2 * br * n * sizeof(double2) + (size_t)(2 * SJ64_BRMAX) * (2 * SJ64_BRMAX) * sizeof(double2);
}

__global__ void __launch_bounds__(SJ64_NT, 1) k_sj64_sweeps(double2* R, double2* Jt, int n, int br, int nb,
                                                            double tol, Sj64Ctl* ctl, unsigned* err) {
  extern __shared__ __align__(16) unsigned char sj64_sm[];
  double2* X = reinterpret_cast<double2*>(sj64_sm);            // [2 br][n]
  double2* Wm = X + (size_t)2 * br * n;                         // [2 br][2 br]
  __shared__ double red[SJ64_BRMAX][SJ64_WPP][2];               // per pair slot and warp: g
  __shared__ double nrm[2 * SJ64_BRMAX];                        // ||row||^2 of the rows held
  __shared__ unsigned s_cnt, s_vis;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int quad = warp / SJ64_WPP, qw = warp % SJ64_WPP;
  const int qt = qw * 32 + lane;
  const int nbp = (nb % 2) ? nb + 1 : nb;

  auto visit = [&](int nrow, bool cross, auto grow) {
    for (int idx = tid; idx < nrow * n; idx += SJ64_NT) {
      const int a = idx / n, o = idx - a * n;
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                       (unsigned)__cvta_generic_to_shared(X + (size_t)a * n + o)),
                   "l"(R + (long long)grow(a) * n + o)
                   : "memory");
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    for (int e = tid; e < nrow * nrow; e += SJ64_NT) Wm[e] = make_double2(e / nrow == e % nrow ? 1.0 : 0.0, 0.0);
    if (tid == 0) s_vis = 0;
    __syncthreads();
    for (int a = warp; a < nrow; a += SJ64_NT / 32) {
      const double2* xr = X + (size_t)a * n;
      double f = 0.0;
      for (int i = lane; i < n; i += 32) f = fma(xr[i].x, xr[i].x, fma(xr[i].y, xr[i].y, f));
      f = warp_sum_d(f);
      if (lane == 0) nrm[a] = f;
    }
    __syncthreads();
    const int rounds = cross ? br : nrow - 1;
    const int pairs = cross ? br : nrow / 2;
    for (int ir = 0; ir < rounds; ++ir) {
      if (quad < pairs) {
        int a, b;
        if (cross) { a = quad; b = br + (quad + ir) % br; }
        else pair_of(ir, quad, nrow, a, b);
        double2* xa = X + (size_t)a * n;
        double2* xb = X + (size_t)b * n;
        double gr = 0.0, gi = 0.0;  // g = row_a . conj(row_b)
        for (int i = qt; i < n; i += 32 * SJ64_WPP) {
          const double2 x = xa[i], y = xb[i];
          gr = fma(x.x, y.x, fma(x.y, y.y, gr));
          gi = fma(x.y, y.x, fma(-x.x, y.y, gi));
        }
        gr = warp_sum_d(gr);
        gi = warp_sum_d(gi);
        if (lane == 0) { red[quad][qw][0] = gr; red[quad][qw][1] = gi; }
        asm volatile("bar.sync %0, %1;" ::"r"(1 + quad), "n"(32 * SJ64_WPP) : "memory");
        gr = red[quad][0][0];
        gi = red[quad][0][1];
#pragma unroll
        for (int w = 1; w < SJ64_WPP; ++w) { gr += red[quad][w][0]; gi += red[quad][w][1]; }
        const double A = nrm[a], B = nrm[b];
        const double ab = hypot(gr, gi);
        if (ab > 1e-300 && ab > tol * sqrt(A) * sqrt(B)) {  // slot-uniform
          const double inv = 1.0 / ab;
          const double z = (B - A) * (0.5 * inv);
          const double t = fabs(z) > 1e150 ? 0.5 / z : copysign(1.0, z) / (fabs(z) + sqrt(fma(z, z, 1.0)));
          const double qq = sqrt(fma(t, t, 1.0));
          const double c = 1.0 - (t * t) / (qq * (1.0 + qq)), sn = t * c;
          const double er = sn * (gr * inv), ei = sn * (gi * inv);
          for (int j2 = qt; j2 < n; j2 += 32 * SJ64_WPP) {
            const double2 x = xa[j2], y = xb[j2];
            xa[j2] = make_double2(c * x.x - (er * y.x - ei * y.y), c * x.y - (er * y.y + ei * y.x));
            xb[j2] = make_double2((er * x.x + ei * x.y) + c * y.x, (er * x.y - ei * x.x) + c * y.y);
          }
          if (qw == 0) {
            if (lane < nrow) {
              const double2 x = Wm[a * nrow + lane], y = Wm[b * nrow + lane];
              Wm[a * nrow + lane] = make_double2(c * x.x - (er * y.x - ei * y.y), c * x.y - (er * y.y + ei * y.x));
              Wm[b * nrow + lane] = make_double2((er * x.x + ei * x.y) + c * y.x, (er * x.y - ei * x.x) + c * y.y);
            }
            if (lane == 0) {
              atomicAdd(&s_vis, 1u);
              nrm[a] = A - t * ab;
              nrm[b] = B + t * ab;
            }
          }
        }
      }
      __syncthreads();
    }
    if (s_vis) {
      for (int idx = tid; idx < nrow * n; idx += SJ64_NT) {
        const int a = idx / n, o = idx - a * n;
        R[(long long)grow(a) * n + o] = X[(size_t)a * n + o];
      }
      for (int cc = tid; cc < n; cc += SJ64_NT) {
        double2 in[2 * SJ64_BRMAX];
#pragma unroll
        for (int a = 0; a < 2 * SJ64_BRMAX; ++a)
          if (a < nrow) in[a] = __ldcg(Jt + (long long)grow(a) * n + cc);
#pragma unroll
        for (int a = 0; a < 2 * SJ64_BRMAX; ++a) {
          if (a < nrow) {
            double2 o = make_double2(0.0, 0.0);
#pragma unroll
            for (int b = 0; b < 2 * SJ64_BRMAX; ++b) {
              if (b < nrow) {
                const double2 wv = Wm[a * nrow + b];
                o.x = fma(wv.x, in[b].x, fma(-wv.y, in[b].y, o.x));
                o.y = fma(wv.x, in[b].y, fma(wv.y, in[b].x, o.y));
              }
            }
            Jt[(long long)grow(a) * n + cc] = o;
          }
        }
      }
      if (tid == 0) s_cnt += s_vis;
    }
    __syncthreads();
  };

  for (int sweep = 0; sweep < SJ64_MAX_SWEEPS; ++sweep) {
    if (tid == 0) s_cnt = 0;
    if (br > 1) {
      for (int blk = blockIdx.x; blk < nb; blk += gridDim.x)
        visit(br, false, [&](int a) { return blk * br + a; });
      if (!grid_barrier(ctl->bar, gridDim.x, err)) return;
    }
    for (int r = 0; r < nbp - 1; ++r) {
      for (int k = blockIdx.x; k < nbp / 2; k += gridDim.x) {
        int P, Q;
        pair_of(r, k, nbp, P, Q);
        if (Q < nb)
          visit(2 * br, true, [&](int a) { return a < br ? P * br + a : Q * br + (a - br); });
      }
      if (!grid_barrier(ctl->bar, gridDim.x, err)) return;
    }
    if (tid == 0 && s_cnt) atomicAdd(&ctl->rot[sweep], s_cnt);
    if (!grid_barrier(ctl->bar, gridDim.x, err)) return;
    if (*reinterpret_cast<volatile unsigned*>(&ctl->rot[sweep]) == 0) {
      if (blockIdx.x == 0 && tid == 0) ctl->sweeps = sweep + 1;
      return;
    }
  }
  if (blockIdx.x == 0 && tid == 0) ctl->sweeps = SJ64_MAX_SWEEPS + 1;
}

__global__ void k_eye64_ld(double2* J, int n, int ld) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)n * n) return;
  const long long r = idx / n, c = idx % n;
  J[r * ld + c] = make_double2(r == c ? 1.0 : 0.0, 0.0);
}

// s2[i] = ||r_i||^2 / ||j_i||^2, jn[i] = 1 / ||j_i||, one warp per row (the ratio cancels the
// drift of a row's norm under rotations that are unitary only to rounding)
__global__ void k_sj64_norms(const double2* R, const double2* Jt, int n, int ld, double* s2, double* jn) {
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (row >= n) return;
  double acc = 0.0, accj = 0.0;
  for (int i = lane; i < n; i += 32) {
    const double2 x = R[(long long)row * ld + i], y = Jt[(long long)row * ld + i];
    acc = fma(x.x, x.x, fma(x.y, x.y, acc));
    accj = fma(y.x, y.x, fma(y.y, y.y, accj));
  }
  acc = warp_sum_d(acc);
  accj = warp_sum_d(accj);
  if (lane == 0) {
    s2[row] = accj > 0 ? acc / accj : acc;
    jn[row] = accj > 0 ? 1.0 / sqrt(accj) : 1.0;
  }
}

__global__ void k_sj64_gather(const double2* Jt, const int* order, const double* jn, int n, int ld,
                              double2* Vh, unsigned* err) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)n * n) return;
  const int r = (int)(idx / n), c = (int)(idx % n);
  const int src = order[r];
  if (src < 0 || src >= n) {
    if (c == 0) atomicOr(err, DEVERR_BOUNDS);
    return;
  }
  const double2 v = Jt[(long long)src * ld + c];
  const double f = jn[src];
  Vh[idx] = make_double2(f * v.x, f * v.y);
}

int sj64_rows_per_block(int n) {
  for (int br = SJ64_BRMAX; br > 1; br /= 2)
    if (sj64_smem_bytes(n, br) <= 200 * 1024) return br;
  return sj64_smem_bytes(n, 1) <= 220 * 1024 ? 1 : 0;
}

int sj64_grid(int npairs, size_t smem) {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sj64_sweeps, SJ64_NT, smem) != cudaSuccess)
    return 0;
  return std::min(npairs, std::min(sms * per, 2 * sms));
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

bool svd64_supported(int n) { return n >= 1 && sj64_rows_per_block(n + (n & 1)) >= 1; }

size_t svd64_work_bytes(int n) {
  const int ld = n + (n & 1);
  const int br = std::max(1, sj64_rows_per_block(ld));
  const size_t rows = (size_t)ceil_div(n, br) * br;
  return align_up(2 * rows * ld * sizeof(double2), 256) + align_up((size_t)n * sizeof(double), 256) +
         align_up((size_t)n * sizeof(int), 256) + align_up(sizeof(Sj64Ctl), 256) +
         align_up((size_t)n * sizeof(double), 256);
}

int svd_rows_jacobi64(const double2* Rz, long long ldr, int n, double* w, double2* Vh, void* work,
                      size_t work_bytes, cudaStream_t st, unsigned* err, int* sweeps) {
  if (n < 1 || ldr < n || !Rz || !w || !Vh || !work || work_bytes < svd64_work_bytes(n))
    return QRTEBD_ERR_INVALID_ARG;
  const int ld = n + (n & 1);
  const int br = sj64_rows_per_block(ld);
  if (br < 1) { set_last_message("svd_rows_jacobi64: rows too long for shared memory"); return QRTEBD_ERR_INVALID_ARG; }
  const int nb = (int)ceil_div(n, br);
  const size_t rows = (size_t)nb * br;
  char* q = static_cast<char*>(work);
  double2* R = reinterpret_cast<double2*>(q);
  double2* Jt = R + rows * ld;
  q += align_up(2 * rows * ld * sizeof(double2), 256);
  double* s2 = reinterpret_cast<double*>(q); q += align_up((size_t)n * sizeof(double), 256);
  int* order = reinterpret_cast<int*>(q); q += align_up((size_t)n * sizeof(int), 256);
  Sj64Ctl* ctl = reinterpret_cast<Sj64Ctl*>(q); q += align_up(sizeof(Sj64Ctl), 256);
  double* jn = reinterpret_cast<double*>(q);
  QR_CUDA_TRY(cudaMemsetAsync(R, 0, 2 * rows * ld * sizeof(double2), st));
  QR_CUDA_TRY(cudaMemcpy2DAsync(R, (size_t)ld * sizeof(double2), Rz, (size_t)ldr * sizeof(double2),
                                (size_t)n * sizeof(double2), (size_t)n, cudaMemcpyDeviceToDevice, st));
  k_eye64_ld<<<(unsigned)ceil_div((long long)n * n, 256), 256, 0, st>>>(Jt, n, ld);
  note_launch();
  QR_CUDA_TRY(cudaGetLastError());
  QR_CUDA_TRY(cudaMemsetAsync(ctl, 0, sizeof(Sj64Ctl), st));
  if (n > 1) {
    const size_t smem = sj64_smem_bytes(ld, br);
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] {
      attr = cudaFuncSetAttribute(k_sj64_sweeps, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    });
    QR_CUDA_TRY(attr);
    const int nbp = (nb % 2) ? nb + 1 : nb;
    const int grid = sj64_grid(nbp / 2, smem);
    if (grid < 1) { set_last_message("svd_rows_jacobi64: no resident CTA"); return QRTEBD_ERR_CUDA; }
    // orthogonal to FP64 working accuracy: sqrt(n) eps
    double tol = std::sqrt((double)std::max(n, 16)) * 1.11e-16;
    int nv = ld, brv = br, nbv = nb;
    void* args[] = {&R, &Jt, &nv, &brv, &nbv, &tol, &ctl, &err};
    QR_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_sj64_sweeps, dim3((unsigned)grid), dim3(SJ64_NT),
                                            args, smem, st));
    note_launch();
  }
  k_sj64_norms<<<(unsigned)ceil_div(n, 8), 256, 0, st>>>(R, Jt, n, ld, s2, jn);
  note_launch();
  k_sj_rank<<<(unsigned)ceil_div(n, 128), 128, 0, st>>>(s2, n, w, order);
  note_launch();
  k_sj64_gather<<<(unsigned)ceil_div((long long)n * n, 256), 256, 0, st>>>(Jt, order, jn, n, ld, Vh, err);
  note_launch();
  QR_CUDA_TRY(cudaGetLastError());
  if (sweeps) QR_CUDA_TRY(cudaMemcpyAsync(sweeps, &ctl->sweeps, sizeof(int), cudaMemcpyDeviceToDevice, st));
  return QRTEBD_OK;
}

}  // namespace qrtebd
