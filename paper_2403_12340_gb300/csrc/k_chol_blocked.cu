// Blocked right-looking Cholesky (no pivoting), FP64.
//
// For J = 0, 1, ...: the 64 x 64 diagonal block is factored in shared memory
// by one thread block; the panel below is solved in place by forward
// substitution, one warp per row over every SM; the trailing matrix gets a
// lower SYRK update, which carries nearly all of the O(n^3) work.
//
// With a split-panel buffer (the mixed path) the trailing update runs in
// double-float arithmetic on the FP32 pipes instead: each panel entry is
// stored once as a pair of floats (hi + lo, 48 significant bits), products
// keep their exact FMA error and the cross terms, and the sums carry their
// rounding error in a second float (two-sum), about 2^-46 relative per
// update; the factor itself stays FP64 in memory, and the diagonal blocks
// and panels are FP64.  On this part the FP64 pipe issues one warp
// instruction per 64 cycles per sub-partition and the FP32 pipe one per
// cycle, so twelve FP32 instructions per product still run several times
// faster than one FP64 FMA.
//
// A pivot at or below tol_rel * max(diag) stops the factorisation: the
// first failing column goes to *fail and every later kernel of the sequence
// does nothing.  The caller decides what that means (not positive definite,
// or: fall back to the pivoted factorisation for a rank-deficient C C^T).
#include <algorithm>
#include <atomic>

#include "common.cuh"
#include "kernels.h"

namespace isdf {

constexpr int CB = 64;

__global__ void k_diag_max(const double* __restrict__ W, long long ldw, int n, double* out, int* fail,
                           long long sW = 0) {
  __shared__ double red[256];
  W += sW * blockIdx.x;
  out += blockIdx.x;
  fail += blockIdx.x;
  double m = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, W[i + ldw * (long long)i]);
  red[threadIdx.x] = m;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *out = red[0];
    *fail = -1;
  }
}

// Factor A[j0:j0+bs, j0:j0+bs] (lower part, already updated) in place; the
// strict upper part of the block is zeroed.  One thread block on one SM.
//
// On GB300 a warp's FP64 instruction holds its SM sub-partition for about
// 64 cycles however many of its lanes are active, and one warp's independent
// FP64 instructions do not overlap; the four sub-partitions together finish
// about one warp instruction per 19 cycles.  So the 64 dependent pivots are
// one warp's chain, run alone on its sub-partition, while twelve warps on
// the other three sub-partitions apply the updates one column behind, each
// thread to a fixed set of lower-triangle elements (no index arithmetic in
// the loop; enough warps to hide the shared-memory latency).  The chain
// carries no square root (LDL^T form):
//   iteration j, warp 0:   a_j <- a_j - l_{j-1} a_{j,j-1}   (last update of column j)
//                          r_j = 1 / d_j, d_j = a_jj        (FP32 estimate, two
//                                                           Newton steps r (2 - d r))
//                          l_j = a_j r_j                   (below the diagonal)
//   iteration j, the others: a_k <- a_k - l_{j-1} a_{k,j-1}  for the columns k > j
//   one block barrier per iteration.
// l_j is double buffered, so the chain writes l_j while the others read
// l_{j-1}.  At the end L = A D^-1/2 below the diagonal and D^1/2 on it.
__device__ __forceinline__ double rsqrt_newton(double d) {
  if (!(d > 1e-30 && d < 1e30)) return 1.0 / sqrt(d);  // outside the FP32 range of the first estimate
  double y = (double)rsqrtf((float)d);
  y = y * fma(-0.5 * d * y, y, 1.5);
  return y * fma(-0.5 * d * y, y, 1.5);
}

constexpr int DIAG_THREADS = 512;
constexpr int DIAG_BULK = DIAG_THREADS / 4 * 3;                       // threads of the warps off sub-partition 0
constexpr int DIAG_EPT = (CB * (CB + 1) / 2 + DIAG_BULK - 1) / DIAG_BULK;  // lower-triangle elements per thread

__global__ void __launch_bounds__(DIAG_THREADS) k_chol_diag(double* A, long long lda, int j0, int bs,
                                                           const double* dmax, double tol_rel, int* fail,
                                                           long long sA = 0) {
  __shared__ double Ls[CB][CB + 1];  // Ls[i][k]: the block (lower part), unscaled LDL^T columns
  __shared__ double lc[2][CB];       // l_j and l_{j-1}
  __shared__ double piv[CB];         // d_j
  __shared__ double q[CB];           // d_j^-1/2
  __shared__ int s_bad;
  // problem blockIdx.x of a batch: its matrix, max and flag
  A += sA * blockIdx.x;
  dmax += blockIdx.x;
  fail += blockIdx.x;
  if (*(volatile int*)fail >= 0) return;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  for (int idx = t; idx < CB * CB; idx += blockDim.x) {
    int i = idx & (CB - 1), k = idx >> 6;
    Ls[i][k] = (i < bs && k <= i) ? A[(j0 + i) + lda * (long long)(j0 + k)] : 0.0;
  }
  // the warps on sub-partitions 1-3 own fixed lower-triangle elements (row * 64 + column)
  const bool bulk = (warp & 3) != 0;
  int own[DIAG_EPT];
  {
    const int b = (warp - 1 - (warp >> 2)) * 32 + lane;
#pragma unroll
    for (int q = 0; q < DIAG_EPT; ++q) {
      const int e = b + DIAG_BULK * q;
      own[q] = -1;
      if (bulk && e < CB * (CB + 1) / 2) {
        int a = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
        while ((a + 1) * (a + 2) / 2 <= e) ++a;
        while (a * (a + 1) / 2 > e) --a;
        own[q] = a * CB + (e - a * (a + 1) / 2);
      }
    }
  }
  if (t == 0) s_bad = -1;
  const double thresh = tol_rel * (*dmax);
  __syncthreads();
  for (int j = 0; j < bs; ++j) {
    const double* lp = lc[(j + 1) & 1];  // l_{j-1}
    if (warp == 0) {
      if (j > 0) {
        const double ajj1 = Ls[j][j - 1];
        for (int i = j + lane; i < bs; i += 32) Ls[i][j] = fma(-lp[i], ajj1, Ls[i][j]);
        __syncwarp();
      }
      const double d = Ls[j][j];
      if (!(d > thresh)) {  // the same value in every lane; also catches NaN
        if (lane == 0) s_bad = j;
      } else {
        const double r = recip_newton(d);
        if (lane == 0) piv[j] = d;
        double* lj = lc[j & 1];
        for (int i = j + 1 + lane; i < bs; i += 32) lj[i] = Ls[i][j] * r;
      }
    } else if (bulk && j > 0) {
      // column j-1 applied to the owned elements of the columns k > j
#pragma unroll
      for (int q = 0; q < DIAG_EPT; ++q) {
        const int o = own[q];
        const int i = o >> 6, k = o & (CB - 1);
        if (o >= 0 && k > j && i < bs) Ls[i][k] = fma(-lp[i], Ls[k][j - 1], Ls[i][k]);
      }
    }
    __syncthreads();
    if (s_bad >= 0) break;
  }
  if (s_bad >= 0) {
    if (t == 0) atomicCAS(fail, -1, j0 + s_bad);
    return;
  }
  if (t < bs) q[t] = rsqrt_newton(piv[t]);
  __syncthreads();
  for (int idx = t; idx < bs * bs; idx += blockDim.x) {
    const int i = idx % bs, k = idx / bs;
    const double v = (k < i) ? Ls[i][k] * q[k] : (k == i ? piv[i] * q[i] : 0.0);
    A[(j0 + i) + lda * (long long)(j0 + k)] = v;
  }
}

// k_chol_diag in double-float arithmetic on the FP32 pipe (the mixed path),
// blocked, which also inverts the factor of the block.  Every element is a
// float pair (about 2^-47 relative per operation); the block is padded to
// 64 x 64 with the identity, so padded pivots are 1 and padded rows of the
// factor are 0.  A = Lt D Lt^T (Lt unit lower) by eight panels of eight
// columns with look-ahead:
//  - warp 0 factors a panel: for each pivot j, d_j = A_jj (accepted when its
//    high part exceeds tol_rel * max diag, in FP32), u_ij = A_ij and
//    l_ij = u_ij / d_j for the rows below, then the rest of the panel's
//    columns take the rank-1 update A_ik -= l_ij u_kj (lanes own rows,
//    __syncwarp between the steps; one warp's chain, no block barrier);
//  - the other warps meanwhile apply the previous panel's rank-8 update to
//    the columns beyond the panel being factored (8 x 8 element blocks of
//    the lower triangle, eight double-float products per element);
//  - between panels all warps update the next panel's columns first, so
//    warp 0 can start on it at once.
// Then B = Lt^-1 by 8 x 8 block rows (diagonal blocks by forward
// substitution, one thread per column; off-diagonal blocks
// B_IJ = -B_II sum_K Lt_IK B_KJ), L = Lt D^1/2 back to A in FP64 and
// L^-1 = D^-1/2 B to Lid (FP64, ld ldi) and / or Lis (float pairs, ld lds).
// Entries are split into float pairs as they are loaded.
constexpr int DF_DIAG_THREADS = 256;
constexpr int DF_PW = 8;  // panel width

// 8 x 8 element block (bi, bk) of the lower triangle, bk <= bi: the block
// count of rows 0..n-1 is n (n + 1) / 2; decode by a short search (n <= 8)
__device__ __forceinline__ void df_tri_block(int b, int& bi, int& bk) {
  int i = 0;
  while ((i + 1) * (i + 2) / 2 <= b) ++i;
  bi = i;
  bk = b - i * (i + 1) / 2;
}

__global__ void __launch_bounds__(DF_DIAG_THREADS) k_chol_diag_df(double* A, long long lda, int j0, int bs,
                                                                 const double* dmax, double tol_rel, int* fail,
                                                                 long long sA, double* Lid, long long ldi,
                                                                 float2* Lis, long long lds, long long sS) {
  __shared__ float2 Ls[CB][CB + 1];     // the block; after its panel, column j holds l_ij (i > j)
  __shared__ float2 Bs[CB][CB + 1];     // B = Lt^-1
  __shared__ float2 Us[2][CB][DF_PW];   // u_kj = l_kj d_j of the last two panels
  __shared__ float2 piv[CB];            // d_j
  __shared__ float2 sq[2][CB];          // d^-1/2, d^1/2
  __shared__ int s_bad;
  A += sA * blockIdx.x;
  dmax += blockIdx.x;
  fail += blockIdx.x;
  if (*(volatile int*)fail >= 0) return;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  for (int idx = t; idx < CB * CB; idx += blockDim.x) {
    const int i = idx & (CB - 1), k = idx >> 6;
    float2 v = make_float2(i == k ? 1.0f : 0.0f, 0.0f);  // the identity beyond bs
    if (i < bs && k < bs) v = k <= i ? split_f64_fast(A[(j0 + i) + lda * (long long)(j0 + k)]) : make_float2(0.f, 0.f);
    Ls[i][k] = v;
    Bs[i][k] = make_float2(0.0f, 0.0f);
  }
  if (t == 0) s_bad = -1;
  const float thresh = (float)(tol_rel * (*dmax));
  __syncthreads();

  // rank-8 update by panel p (l in Ls columns c0..c0+7, u in Us[p & 1]) of
  // the lower-triangle 8 x 8 blocks with block column in [kb0, kb1): thread
  // `tid` of `nth`
  auto update_blocks = [&](int p, int kb0, int kb1, int tid, int nth) {
    const int c0 = p * DF_PW;
    const float2(*U)[DF_PW] = Us[p & 1];
    // blocks (bi, bk) with kb0 <= bk < kb1 and bk <= bi < 8
    int nblk = 0;
    for (int bk = kb0; bk < kb1; ++bk) nblk += 8 - bk;
    for (int e = tid; e < nblk * 64; e += nth) {
      int b = e >> 6, bi = 0, bk = kb0;
      while (b >= 8 - bk) {
        b -= 8 - bk;
        ++bk;
      }
      bi = bk + b;
      const int i = bi * 8 + ((e >> 3) & 7), k = bk * 8 + (e & 7);
      if (k > i) continue;
      float hi = Ls[i][k].x, lo = Ls[i][k].y;
#pragma unroll
      for (int q = 0; q < DF_PW; ++q) {
        const float2 l = Ls[i][c0 + q];
        df_fma(make_float2(-l.x, -l.y), U[k][q], hi, lo);
      }
      Ls[i][k] = df_norm(hi, lo);
    }
  };

  constexpr int NP = CB / DF_PW;
  for (int p = 0; p < NP; ++p) {
    const int c0 = p * DF_PW;
    if (warp == 0) {
      // ---- panel p in registers: lane owns rows c0 + lane and c0 + 32 + lane
      // (v[0], v[1]), columns c0..c0+7; row j = c0 + jq is lane jq's v[0]
      float2(*U)[DF_PW] = Us[p & 1];
      float2 v[2][DF_PW];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int i = c0 + lane + 32 * h;
#pragma unroll
        for (int q = 0; q < DF_PW; ++q) v[h][q] = i < CB ? Ls[i][c0 + q] : make_float2(0.f, 0.f);
      }
      bool bad = false;
#pragma unroll
      for (int jq = 0; jq < DF_PW; ++jq) {
        const int j = c0 + jq;
        float2 d;
        d.x = __shfl_sync(0xffffffffu, v[0][jq].x, jq);
        d.y = __shfl_sync(0xffffffffu, v[0][jq].y, jq);
        // u_kj = A_kj of the panel's later rows k = c0 + kq, before scaling
        float2 uk[DF_PW];
#pragma unroll
        for (int kq = jq + 1; kq < DF_PW; ++kq) {
          uk[kq].x = __shfl_sync(0xffffffffu, v[0][jq].x, kq);
          uk[kq].y = __shfl_sync(0xffffffffu, v[0][jq].y, kq);
        }
        if (!bad) {
          if (j < bs && !(d.x > thresh)) {  // the same value in every lane; also catches NaN
            bad = true;
            if (lane == 0) s_bad = j;
          } else {
            const float2 r = df_recip(d);
            if (lane == 0) piv[j] = d;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int i = c0 + lane + 32 * h;
              if (i > j && i < CB) {
                const float2 u = v[h][jq];
                U[i][jq] = u;
                const float2 l = df_mul(u, r);
                v[h][jq] = l;
#pragma unroll
                for (int kq = jq + 1; kq < DF_PW; ++kq)
                  if (c0 + kq <= i) v[h][kq] = df_fms(v[h][kq], l, uk[kq]);
              }
            }
          }
        }
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int i = c0 + lane + 32 * h;
        if (i < CB) {
#pragma unroll
          for (int q = 0; q < DF_PW; ++q) Ls[i][c0 + q] = v[h][q];
        }
      }
    } else if (p > 0 && (warp & 3) != 0) {
      // ---- the previous panel's update of the columns beyond this panel, by
      // the warps off warp 0's sub-partition (the chain keeps its issue slots)
      update_blocks(p - 1, p + 1, NP, (warp - 1 - (warp >> 2)) * 32 + lane, DF_DIAG_THREADS / 4 * 3);
    }
    __syncthreads();
    if (s_bad >= 0) break;
    // ---- this panel's update of the next panel's columns (look-ahead)
    if (p + 1 < NP) update_blocks(p, p + 1, p + 2, t, DF_DIAG_THREADS);
    __syncthreads();
  }
  if (s_bad >= 0) {
    if (t == 0) atomicCAS(fail, -1, j0 + s_bad);
    return;
  }
  // ---- B = Lt^-1: diagonal 8 x 8 blocks, one thread per column
  if (t < CB) {
    const int bi = t >> 3, m = t;  // column m of diagonal block bi
    Bs[m][m] = make_float2(1.0f, 0.0f);
    for (int i = m + 1; i < bi * 8 + 8; ++i) {
      float hi = 0.0f, lo = 0.0f;
      for (int j = m; j < i; ++j) df_fma(Ls[i][j], Bs[j][m], hi, lo);
      Bs[i][m] = df_norm(-hi, -lo);
    }
  }
  __syncthreads();
  // off-diagonal blocks, block row by block row: W = sum_K Lt_IK B_KJ
  // (K = J .. I - 1, into the block itself), then B_IJ = -B_II W
  for (int I = 1; I < NP; ++I) {
    float2 w[2];
    int cnt = 0;
    for (int e = t; e < I * 64; e += blockDim.x, ++cnt) {
      const int J = e >> 6, i = I * 8 + ((e >> 3) & 7), m = J * 8 + (e & 7);
      // two interleaved sums halve the dependent chain
      float hi = 0.0f, lo = 0.0f, hi2 = 0.0f, lo2 = 0.0f;
      int j = m;
      for (; j + 1 < I * 8; j += 2) {
        df_fma(Ls[i][j], Bs[j][m], hi, lo);
        df_fma(Ls[i][j + 1], Bs[j + 1][m], hi2, lo2);
      }
      if (j < I * 8) df_fma(Ls[i][j], Bs[j][m], hi, lo);
      df_fma(make_float2(hi2, lo2), make_float2(1.0f, 0.0f), hi, lo);
      w[cnt] = df_norm(hi, lo);
    }
    cnt = 0;
    for (int e = t; e < I * 64; e += blockDim.x, ++cnt) {
      const int i = I * 8 + ((e >> 3) & 7), m = (e >> 6) * 8 + (e & 7);
      Bs[i][m] = w[cnt];
    }
    __syncthreads();
    cnt = 0;
    for (int e = t; e < I * 64; e += blockDim.x, ++cnt) {
      const int i = I * 8 + ((e >> 3) & 7), m = (e >> 6) * 8 + (e & 7);
      float hi = 0.0f, lo = 0.0f;
      for (int j = I * 8; j <= i; ++j) df_fma(Bs[i][j], Bs[j][m], hi, lo);  // B_II W (B_ii = 1)
      w[cnt] = df_norm(-hi, -lo);
    }
    __syncthreads();
    cnt = 0;
    for (int e = t; e < I * 64; e += blockDim.x, ++cnt) {
      const int i = I * 8 + ((e >> 3) & 7), m = (e >> 6) * 8 + (e & 7);
      Bs[i][m] = w[cnt];
    }
    __syncthreads();
  }
  // ---- L = Lt D^1/2, L^-1 = D^-1/2 B
  if (t < bs) {
    const float2 dq = df_rsqrt(piv[t]);
    sq[0][t] = dq;
    sq[1][t] = df_mul(piv[t], dq);
  }
  __syncthreads();
  for (int idx = t; idx < bs * bs; idx += blockDim.x) {
    const int i = idx % bs, k = idx / bs;
    const double v = (k < i) ? df_to_f64(df_mul(Ls[i][k], sq[1][k])) : (k == i ? df_to_f64(sq[1][i]) : 0.0);
    A[(j0 + i) + lda * (long long)(j0 + k)] = v;
    if (Lid || Lis) {
      const float2 w = (k < i) ? df_mul(Bs[i][k], sq[0][i]) : (k == i ? sq[0][i] : make_float2(0.0f, 0.0f));
      if (Lid) Lid[i + ldi * (long long)k] = df_to_f64(w);
      if (Lis) Lis[sS * blockIdx.x + i + lds * k] = w;
    }
  }
}

// The panel below a factored diagonal block, A21 <- A21 L_jj^-T, in place:
// one warp per row, lane l holding columns l and l + 32 of the row; forward
// substitution by columns, each solved value broadcast by a shuffle.  Rows
// are independent, so every SM takes part however short the panel is.
// With Sp, the solved panel is also written as float pairs: row `row` of
// the panel, column c at Sp[row + lds c] (problem y at Sp + y sS).
__global__ void __launch_bounds__(256) k_panel_trsm(double* A, long long lda, int j0, int bs, int rem,
                                                   const int* fail, long long sA = 0, float2* Sp = nullptr,
                                                   long long lds = 0, long long sS = 0) {
  __shared__ double Lt[CB][CB + 1];  // Lt[c][k] = L_jj(c, k), zero outside the lower triangle
  __shared__ double inv[CB];
  A += sA * blockIdx.y;  // problem blockIdx.y of a batch
  if (*(volatile const int*)(fail + blockIdx.y) >= 0) return;
  const int t = threadIdx.x;
  for (int idx = t; idx < CB * CB; idx += blockDim.x) {
    const int i = idx & (CB - 1), k = idx >> 6;
    Lt[i][k] = (i < bs && k <= i) ? A[(j0 + i) + lda * (long long)(j0 + k)] : 0.0;
  }
  __syncthreads();
  if (t < bs) inv[t] = 1.0 / Lt[t][t];
  __syncthreads();
  const int warp = t >> 5, lane = t & 31;
  for (int row = blockIdx.x * 8 + warp; row < rem; row += gridDim.x * 8) {
    double* a = A + (j0 + bs + row) + lda * (long long)j0;
    double x0 = lane < bs ? a[lda * lane] : 0.0;
    double x1 = lane + 32 < bs ? a[lda * (lane + 32)] : 0.0;
    for (int k = 0; k < bs; ++k) {
      double xk;
      if (k < 32) {
        if (lane == k) x0 *= inv[k];
        xk = __shfl_sync(0xffffffffu, x0, k);
      } else {
        if (lane == k - 32) x1 *= inv[k];
        xk = __shfl_sync(0xffffffffu, x1, k - 32);
      }
      if (lane > k) x0 = fma(-xk, Lt[lane][k], x0);
      if (lane + 32 > k) x1 = fma(-xk, Lt[lane + 32][k], x1);
    }
    if (lane < bs) a[lda * lane] = x0;
    if (lane + 32 < bs) a[lda * (lane + 32)] = x1;
    if (Sp) {
      float2* sp = Sp + sS * blockIdx.y + row;
      if (lane < bs) sp[lds * lane] = split_f64(x0);
      if (lane + 32 < bs) sp[lds * (lane + 32)] = split_f64(x1);
    }
  }
}

// The panel of the mixed path as a product, A21 <- A21 L_jj^-T, with the
// float pairs of L_jj^-1 that k_chol_diag_df wrote (Lis, ld lds): each
// output is an independent dot product, so no substitution chain remains.
// One block per 16 panel rows (256 threads, a row and four columns each),
// double-float accumulation on the FP32 pipe; rows are read whole into
// shared memory before any is written back, in FP64 to A and as the float
// pairs of the split panel Sp for the trailing update.
constexpr int PG_ROWS = 16;

__global__ void __launch_bounds__(256) k_panel_gemm_df(double* A, long long lda, int j0, int bs, int rem,
                                                      const int* fail, long long sA, float2* Sp, long long lds,
                                                      long long sS, const float2* __restrict__ Lis) {
  __shared__ float2 As[PG_ROWS][CB + 1];
  __shared__ float2 Bs[CB][CB + 1];  // Bs[j][m] = (L_jj^-1)(j, m), zero above the diagonal
  A += sA * blockIdx.y;
  Sp += sS * blockIdx.y;
  Lis += sS * blockIdx.y;
  if (*(volatile const int*)(fail + blockIdx.y) >= 0) return;
  const int t = threadIdx.x;
  const int row0 = blockIdx.x * PG_ROWS;
  const float2 zero = make_float2(0.0f, 0.0f);
  for (int idx = t; idx < CB * CB; idx += blockDim.x) {
    const int jj = idx & (CB - 1), m = idx >> 6;
    Bs[jj][m] = (jj < bs && m <= jj) ? Lis[jj + lds * m] : zero;
  }
  for (int idx = t; idx < PG_ROWS * CB; idx += blockDim.x) {
    const int rr = idx % PG_ROWS, m = idx / PG_ROWS;
    const int row = row0 + rr;
    As[rr][m] = (row < rem && m < bs) ? split_f64_fast(A[(j0 + bs + row) + lda * (long long)(j0 + m)]) : zero;
  }
  __syncthreads();
  const int rr = t >> 4, cq = t & 15;
  float hi[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f};
  for (int m0 = 0; m0 < bs; m0 += 32) {
    const int me = min(bs, m0 + 32);
    for (int m = m0; m < me; ++m) {
      const float2 a = As[rr][m];
#pragma unroll
      for (int q = 0; q < 4; ++q) df_fma(a, Bs[cq + 16 * q][m], hi[q], lo[q]);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) df_renorm(hi[q], lo[q]);
  }
  const int row = row0 + rr;
  if (row >= rem) return;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int jj = cq + 16 * q;
    if (jj >= bs) continue;
    const float2 x = df_norm(hi[q], lo[q]);
    A[(j0 + bs + row) + lda * (long long)(j0 + jj)] = df_to_f64(x);
    Sp[row + lds * jj] = x;
  }
}

// Zero the strict upper triangle (matrix blockIdx.z at A + z sA).
__global__ void k_zero_upper(double* A, long long lda, int n, long long sA = 0) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int k = blockIdx.y;
  A += sA * blockIdx.z;
  if (i < k && k < n) A[i + lda * (long long)k] = 0.0;
}

// dst(i, j) = src(i, j) for i < rows, j < cols; problem blockIdx.z at
// dst + z sD, src + z sS
__global__ void k_copy_block(const double* __restrict__ src, long long lds, long long sS, double* __restrict__ dst,
                             long long ldd, long long sD, int rows, int cols) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i < rows && j < cols) dst[sD * blockIdx.z + i + ldd * j] = src[sS * blockIdx.z + i + lds * j];
}

// The trailing update of one step, A22 <- A22 - P P^T over the lower tiles
// of A22, P = L[j0 + bs :, j0 : j0 + bs] the solved panel (K = bs <= 64):
// one TS x TS output tile per block, (TS / 4)^2 threads with a 4 x 4
// register tile each, strided by TS / 4 so that the shared-memory reads of a
// warp hit consecutive words; the panel rows of the tile go through shared
// memory in K chunks of 32.  Every thread issues only FP64 FMAs in the inner
// loop, 16 per pair of 4-element reads.  The strict upper triangle of a
// diagonal tile is left alone (only the lower triangle is ever read).
// Problem blockIdx.y of a batch at L + y sL.
template <int TS, int TM>
__global__ void __launch_bounds__((TS / TM) * (TS / TM)) k_trail_update(double* L, long long ldl, int j0, int bs,
                                                                       int rem, const int* fail, long long sL) {
  constexpr int Q = TS / TM, NT = Q * Q, KC = 32;
  __shared__ double As[KC][TS], Bs[KC][TS];
  L += sL * blockIdx.y;
  if (*(volatile const int*)(fail + blockIdx.y) >= 0) return;
  const int tile = blockIdx.x;
  int ti = (int)((sqrtf(8.0f * (float)tile + 1.0f) - 1.0f) * 0.5f);
  while ((ti + 1) * (ti + 2) / 2 <= tile) ++ti;
  while (ti * (ti + 1) / 2 > tile) --ti;
  const int tj = tile - ti * (ti + 1) / 2;
  const int i0 = ti * TS, k0 = tj * TS;  // tile origin inside the trailing block
  const int t = threadIdx.x, tx = t % Q, ty = t / Q;
  const long long r0 = j0 + bs;
  const double* P = L + r0 + ldl * (long long)j0;  // P(i, c) at P[i + ldl c]
  double acc[TM][TM];
#pragma unroll
  for (int m = 0; m < TM; ++m)
#pragma unroll
    for (int n = 0; n < TM; ++n) acc[m][n] = 0.0;
  for (int c0 = 0; c0 < bs; c0 += KC) {
    const int kc = min(KC, bs - c0);
    for (int idx = t; idx < KC * TS; idx += NT) {
      const int i = idx % TS, c = idx / TS;
      const bool in_k = c < kc;
      As[c][i] = (in_k && i0 + i < rem) ? P[(i0 + i) + ldl * (long long)(c0 + c)] : 0.0;
      Bs[c][i] = (in_k && k0 + i < rem) ? P[(k0 + i) + ldl * (long long)(c0 + c)] : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int c = 0; c < KC; ++c) {
      double a[TM], b[TM];
#pragma unroll
      for (int m = 0; m < TM; ++m) {
        a[m] = As[c][tx + Q * m];
        b[m] = Bs[c][ty + Q * m];
      }
#pragma unroll
      for (int m = 0; m < TM; ++m)
#pragma unroll
        for (int n = 0; n < TM; ++n) acc[m][n] = fma(a[m], b[n], acc[m][n]);
    }
    __syncthreads();
  }
  double* C = L + r0 + ldl * r0;
#pragma unroll
  for (int m = 0; m < TM; ++m)
#pragma unroll
    for (int n = 0; n < TM; ++n) {
      const int i = i0 + tx + Q * m, k = k0 + ty + Q * n;
      if (i < rem && k < rem && (ti != tj || i >= k)) C[i + ldl * (long long)k] -= acc[m][n];
    }
}

// The same trailing update in double-float arithmetic from the split panel
// Sp (rows of the panel, ld lds, problem y at Sp + y sS): FP32 shared tiles
// of float pairs, a (hi, lo) accumulator pair per output, renormalised after
// every K chunk; C -= hi + lo in FP64 at the end.
template <int TS, int TM>
// tj0 > 0 or tj1 < T (T tiles per side): only the tile columns [tj0, tj1)
// of the trailing triangle, enumerated column by column (the look-ahead of
// launch_cholesky_and_inverse splits one update in two).
__global__ void __launch_bounds__((TS / TM) * (TS / TM)) k_trail_update_df(const float2* __restrict__ Sp, long long lds,
                                                                          long long sS, double* L, long long ldl,
                                                                          int j0, int bs, int rem, const int* fail,
                                                                          long long sL, int tj0 = 0, int tj1 = -1) {
  constexpr int Q = TS / TM, NT = Q * Q, KC = 32;
  __shared__ float2 As[KC][TS], Bs[KC][TS];
  L += sL * blockIdx.y;
  Sp += sS * blockIdx.y;
  if (*(volatile const int*)(fail + blockIdx.y) >= 0) return;
  const int tile = blockIdx.x;
  int ti, tj;
  if (tj1 < 0) {
    ti = (int)((sqrtf(8.0f * (float)tile + 1.0f) - 1.0f) * 0.5f);
    while ((ti + 1) * (ti + 2) / 2 <= tile) ++ti;
    while (ti * (ti + 1) / 2 > tile) --ti;
    tj = tile - ti * (ti + 1) / 2;
  } else {
    const int T = (rem + TS - 1) / TS;
    int b = tile;
    tj = tj0;
    while (b >= T - tj) {
      b -= T - tj;
      ++tj;
    }
    ti = tj + b;
  }
  const int i0 = ti * TS, k0 = tj * TS;
  const int t = threadIdx.x, tx = t % Q, ty = t / Q;
  const long long r0 = j0 + bs;
  float hi[TM][TM], lo[TM][TM];
#pragma unroll
  for (int m = 0; m < TM; ++m)
#pragma unroll
    for (int n = 0; n < TM; ++n) hi[m][n] = lo[m][n] = 0.0f;
  for (int c0 = 0; c0 < bs; c0 += KC) {
    const int kc = min(KC, bs - c0);
    for (int idx = t; idx < KC * TS; idx += NT) {
      const int i = idx % TS, c = idx / TS;
      const bool in_k = c < kc;
      As[c][i] = (in_k && i0 + i < rem) ? Sp[(i0 + i) + lds * (c0 + c)] : make_float2(0.0f, 0.0f);
      Bs[c][i] = (in_k && k0 + i < rem) ? Sp[(k0 + i) + lds * (c0 + c)] : make_float2(0.0f, 0.0f);
    }
    __syncthreads();
#pragma unroll 2
    for (int c = 0; c < KC; ++c) {
      float2 a[TM], b[TM];
#pragma unroll
      for (int m = 0; m < TM; ++m) {
        a[m] = As[c][tx + Q * m];
        b[m] = Bs[c][ty + Q * m];
      }
#pragma unroll
      for (int m = 0; m < TM; ++m)
#pragma unroll
        for (int n = 0; n < TM; ++n) df_fma(a[m], b[n], hi[m][n], lo[m][n]);
    }
#pragma unroll
    for (int m = 0; m < TM; ++m)
#pragma unroll
      for (int n = 0; n < TM; ++n) df_renorm(hi[m][n], lo[m][n]);
    __syncthreads();
  }
  double* C = L + r0 + ldl * r0;
#pragma unroll
  for (int m = 0; m < TM; ++m)
#pragma unroll
    for (int n = 0; n < TM; ++n) {
      const int i = i0 + tx + Q * m, k = k0 + ty + Q * n;
      if (i < rem && k < rem && (ti != tj || i >= k))
        C[i + ldl * (long long)k] -= f32_as_f64(hi[m][n]) + f32_as_f64(lo[m][n]);
    }
}

// Tile width of a trailing update: 64 (4 x 4 per thread) while the 64-wide
// tiles fill the SMs, else 32 (2 x 2 per thread, still 256 threads): the
// late, small updates then use four times the SMs, each tile a quarter of
// the work with the same number of warps.
static cudaError_t trail_update(double* L, long long ldl, int j0, int bs, int rem, int batch, const int* fail,
                                long long sL, cudaStream_t s, const float2* Sp = nullptr, long long lds = 0,
                                long long sS = 0) {
  auto tiles = [](int m, int ts) {
    const long long T = (m + ts - 1) / ts;
    return T * (T + 1) / 2;
  };
  static std::atomic<int> sms_cache{0};
  int sms = sms_cache.load(std::memory_order_relaxed);
  if (!sms) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    sms_cache.store(sms, std::memory_order_relaxed);
  }
  KernelTimer kt(Sp ? KF_DF_GEMM : KF_FP64_GEMM, s, (double)rem * (rem + 1) * bs * batch);  // lower triangle, 2 flops per term
  note_launch();
  if (Sp) {
    if (tiles(rem, 64) * batch >= sms) {
      k_trail_update_df<64, 4><<<dim3((unsigned)tiles(rem, 64), batch), 256, 0, s>>>(Sp, lds, sS, L, ldl, j0, bs,
                                                                                     rem, fail, sL);
    } else {
      k_trail_update_df<32, 2><<<dim3((unsigned)tiles(rem, 32), batch), 256, 0, s>>>(Sp, lds, sS, L, ldl, j0, bs,
                                                                                     rem, fail, sL);
    }
  } else if (tiles(rem, 64) * batch >= sms) {
    k_trail_update<64, 4><<<dim3((unsigned)tiles(rem, 64), batch), 256, 0, s>>>(L, ldl, j0, bs, rem, fail, sL);
  } else {
    k_trail_update<32, 2><<<dim3((unsigned)tiles(rem, 32), batch), 256, 0, s>>>(L, ldl, j0, bs, rem, fail, sL);
  }
  return cudaGetLastError();
}

// Double-float trailing update of one column range of the trailing block:
// part 1 the first 64 columns (the next diagonal block and its panel),
// part 2 the rest (see launch_cholesky_and_inverse).
static cudaError_t trail_update_part(double* L, long long ldl, int j0, int bs, int rem, const int* fail,
                                     cudaStream_t s, const float2* Sp, long long lds, int part) {
  if (rem <= 0) return cudaSuccess;
  constexpr int TS = 32;  // the thin first part needs the parallelism; the rest follows the full rule below
  const int T = (rem + TS - 1) / TS, split = std::min(T, CB / TS);
  const int tj0 = part == 1 ? 0 : split, tj1 = part == 1 ? split : T;
  if (tj0 >= tj1) return cudaSuccess;
  long long ntiles = 0;
  for (int tj = tj0; tj < tj1; ++tj) ntiles += T - tj;
  const long long cols0 = (long long)tj0 * TS, cols1 = std::min<long long>((long long)tj1 * TS, rem);
  // terms: the lower part of columns [cols0, cols1) of the rem x rem triangle, bs each
  const double terms = (double)(cols1 - cols0) * (2.0 * rem - cols0 - cols1 + 1) / 2.0 * bs;
  KernelTimer kt(KF_DF_GEMM, s, 2.0 * terms);
  note_launch();
  if (part == 2 && (T / 2) * (T / 2 + 1) / 2 >= 152) {
    // the wide rest in 64-wide tiles while they fill the GPU (tile columns in 64s)
    const int T64 = (rem + 63) / 64;
    long long n64 = 0;
    for (int tj = 1; tj < T64; ++tj) n64 += T64 - tj;
    k_trail_update_df<64, 4><<<dim3((unsigned)n64, 1), 256, 0, s>>>(Sp, lds, 0, L, ldl, j0, bs, rem, fail, 0, 1, T64);
  } else {
    k_trail_update_df<32, 2><<<dim3((unsigned)ntiles, 1), 256, 0, s>>>(Sp, lds, 0, L, ldl, j0, bs, rem, fail, 0, tj0,
                                                                       tj1);
  }
  return cudaGetLastError();
}

// The mixed path (a split-panel buffer given) factors in double-float
// arithmetic throughout; its rank test then accepts pivots above
// 2^-40 max diag at least (double-float rounding is ~2^-47 per operation, so
// the FP64 threshold of a rank-deficient C C^T could pass noise; a matrix
// that fails here goes to the FP64 pivoted factorisation).
constexpr double kDfPivotTol = 0x1p-40;
static double df_tol(double tol_rel, const float2* split) {
  return split && tol_rel > 0.0 ? std::max(tol_rel, kDfPivotTol) : tol_rel;
}

// One diagonal block.  The mixed path (split != null, split panel of n rows,
// problem z at + z sS) factors in double-float and leaves L_jj^-1 as float
// pairs in the last 64 rows of the split panel, rows that no panel reaches
// (a panel holds at most n - 64 rows); Lid (FP64, ld ldi), if given, gets
// L_jj^-1 too.
static cudaError_t diag_step(double* L, long long ldl, int j0, int bs, const double* dmax, double tol_rel, int* fail,
                             long long sL, int batch, float2* split, long long n, long long sS, double* Lid,
                             long long ldi, cudaStream_t s) {
  KernelTimer kt(KF_CHOL_DIAG, s, bs * (double)bs * bs / 3.0 * batch);  // bs^3 / 3 flops (FP64 or double-float)
  note_launch();
  if (split) {
    float2* lis = n > CB ? split + (n - CB) : nullptr;  // n <= 64: one block, no panel
    k_chol_diag_df<<<batch, DF_DIAG_THREADS, 0, s>>>(L, ldl, j0, bs, dmax, tol_rel, fail, sL, Lid, ldi, lis, n, sS);
  } else {
    k_chol_diag<<<batch, DIAG_THREADS, 0, s>>>(L, ldl, j0, bs, dmax, tol_rel, fail, sL);
  }
  return cudaGetLastError();
}

static unsigned panel_blocks(int rem);

static cudaError_t panel_step(double* L, long long ldl, int j0, int bs, int rem, const int* fail, long long sL,
                              int batch, float2* split, long long lds, long long sS, cudaStream_t s) {
  KernelTimer kt(split ? KF_DF_GEMM : KF_FP64_GEMM, s, (double)rem * bs * bs * batch);  // rem bs^2 flops
  note_launch();
  if (split)
    k_panel_gemm_df<<<dim3((rem + PG_ROWS - 1) / PG_ROWS, batch), 256, 0, s>>>(L, ldl, j0, bs, rem, fail, sL, split,
                                                                              lds, sS, split + (lds - CB));
  else
    k_panel_trsm<<<dim3(panel_blocks(rem), batch), 256, 0, s>>>(L, ldl, j0, bs, rem, fail, sL, nullptr, lds, sS);
  return cudaGetLastError();
}

static unsigned panel_blocks(int rem) {
  const int b = (rem + 7) / 8;
  return (unsigned)(b < 4 * 152 ? b : 4 * 152);
}

cudaError_t launch_cholesky_blocked(const double* W, long long ldw, int n, double tol_rel, double* L, long long ldl,
                                    double* dmax, int* fail, cudaStream_t s, float2* split) {
  if (n <= 0) return cudaSuccess;
  cudaError_t e;
  if (L != W) {
    e = cudaMemcpy2DAsync(L, ldl * sizeof(double), W, ldw * sizeof(double), n * sizeof(double), n,
                          cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
  }
  note_launch();
  k_diag_max<<<1, 256, 0, s>>>(L, ldl, n, dmax, fail);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  tol_rel = df_tol(tol_rel, split);
  for (int j0 = 0; j0 < n; j0 += CB) {
    const int bs = min(CB, n - j0);
    if ((e = diag_step(L, ldl, j0, bs, dmax, tol_rel, fail, 0, 1, split, n, 0, nullptr, 0, s)) != cudaSuccess)
      return e;
    const int rem = n - j0 - bs;
    if (rem <= 0) break;
    if ((e = panel_step(L, ldl, j0, bs, rem, fail, 0, 1, split, n, 0, s)) != cudaSuccess) return e;
    // trailing: A[j0+bs:, j0+bs:] -= L_panel L_panel^T (lower tiles)
    e = trail_update(L, ldl, j0, bs, rem, 1, fail, 0, s, split, n, 0);
    if (e != cudaSuccess) return e;
  }
  dim3 g((n + 127) / 128, n);
  note_launch();
  k_zero_upper<<<g, 128, 0, s>>>(L, ldl, n);
  return cudaGetLastError();
}

cudaError_t launch_cholesky_and_inverse(const double* W, long long ldw, int n, double tol_rel, double* L,
                                        long long ldl, double* Li, long long ldi, double* dmax, int* fail,
                                        double* work, cudaStream_t s, cudaStream_t aux, cudaEvent_t* ev,
                                        float2* split, cudaStream_t aux2) {
  if (n <= 0) return cudaSuccess;
  const int nsteps = (n + CB - 1) / CB;
  const bool ahead = split != nullptr && aux2 != nullptr;
  cudaEvent_t* ev_panel = ev + nsteps;      // panel j written (look-ahead)
  cudaEvent_t* ev_rest = ev + 2 * nsteps;   // rest of update j applied (look-ahead)
  DfGemm df(split != nullptr);  // the inverse rows in the same arithmetic as the trailing updates
  // on s: with double-float blocks the diagonal blocks of Li are written from s
  cudaError_t e = cudaMemset2DAsync(Li, ldi * sizeof(double), 0, n * sizeof(double), n, split ? s : aux);
  if (e != cudaSuccess) return e;
  if (L != W) {
    e = cudaMemcpy2DAsync(L, ldl * sizeof(double), W, ldw * sizeof(double), n * sizeof(double), n,
                          cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
  }
  note_launch();
  k_diag_max<<<1, 256, 0, s>>>(L, ldl, n, dmax, fail);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  double* Y = work;               // 64 x n: L[J, 0:J] Li[0:J, 0:J]
  double* part = work + 64ll * n;  // split-K partials of Y, 8 x 64 x n
  tol_rel = df_tol(tol_rel, split);
  for (int j0 = 0, jb = 0; j0 < n; j0 += CB, ++jb) {
    const int bs = min(CB, n - j0);
    double* Ljj = L + j0 + ldl * (long long)j0;
    double* Lijj = Li + j0 + ldi * (long long)j0;
    // with look-ahead the split panels alternate between two buffers: the
    // rest of step j's update (aux2) still reads panel j while step j + 1
    // writes its own; step j + 2 reuses the buffer after s waited for it
    float2* sp = ahead ? split + (size_t)(jb & 1) * CB * n : split;
    // the double-float block factorisation writes L_jj^-1 into Li itself
    if ((e = diag_step(L, ldl, j0, bs, dmax, tol_rel, fail, 0, 1, sp, n, 0, split ? Lijj : nullptr, ldi, s)) !=
        cudaSuccess)
      return e;
    // row block jb of the inverse, beside the rest of the factorisation
    if ((e = cudaEventRecord(ev[jb], s)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(aux, ev[jb], 0)) != cudaSuccess) return e;
    if (!split && (e = launch_diag_inverse_block(Ljj, ldl, bs, Lijj, ldi, aux)) != cudaSuccess) return e;
    if (j0 > 0) {
      const long long tiles = (long long)((bs + 63) / 64) * ((j0 + 63) / 64);
      const int sp = (int)std::max(1LL, std::min<long long>(8, (2 * 152 + tiles - 1) / tiles));
      e = launch_gemm(L + j0, ldl, false, Li, ldi, true, bs, j0, j0, 1.0, 0.0, Y, bs, false, sp, part, false, aux,
                      TRI_B_LOWER_T);
      if (e != cudaSuccess) return e;
      e = launch_gemm(Lijj, ldi, false, Y, bs, true, bs, j0, bs, -1.0, 0.0, Li + j0, ldi, false, 1, nullptr, false, aux,
                      TRI_A_LOWER);
      if (e != cudaSuccess) return e;
    }
    const int rem = n - j0 - bs;
    if (rem <= 0) break;
    if ((e = panel_step(L, ldl, j0, bs, rem, fail, 0, 1, sp, n, 0, s)) != cudaSuccess) return e;
    if (!ahead) {
      e = trail_update(L, ldl, j0, bs, rem, 1, fail, 0, s, split, n, 0);
      if (e != cudaSuccess) return e;
      continue;
    }
    // look-ahead: the rest of the previous step's update (on aux2) has
    // reached these columns before this step's panel updates them
    if (jb > 0 && (e = cudaStreamWaitEvent(s, ev_rest[jb - 1], 0)) != cudaSuccess) return e;
    if ((e = trail_update_part(L, ldl, j0, bs, rem, fail, s, sp, n, 1)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(ev_panel[jb], s)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(aux2, ev_panel[jb], 0)) != cudaSuccess) return e;
    if ((e = trail_update_part(L, ldl, j0, bs, rem, fail, aux2, sp, n, 2)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(ev_rest[jb], aux2)) != cudaSuccess) return e;
  }
  if (ahead && nsteps > 1 && (e = cudaStreamWaitEvent(s, ev_rest[nsteps - 2], 0)) != cudaSuccess) return e;
  dim3 g((n + 127) / 128, n);
  note_launch();
  k_zero_upper<<<g, 128, 0, s>>>(L, ldl, n);
  return cudaGetLastError();
}

// The same factorisation for `batch` matrices of equal size n (W_z = W + z
// sW, L_z = L + z sL): one launch per step covers every matrix.  dmax and
// fail: batch entries.
cudaError_t launch_cholesky_blocked_batched(const double* W, long long ldw, long long sW, int n, int batch,
                                            double tol_rel, double* L, long long ldl, long long sL, double* dmax,
                                            int* fail, cudaStream_t s, float2* split) {
  if (n <= 0 || batch <= 0) return cudaSuccess;
  if (batch > 65535) return cudaErrorInvalidValue;
  cudaError_t e;
  if (L != W || ldl != ldw || sL != sW) {
    note_launch();
    k_copy_block<<<dim3((n + 127) / 128, n, batch), 128, 0, s>>>(W, ldw, sW, L, ldl, sL, n, n);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  note_launch();
  k_diag_max<<<batch, 256, 0, s>>>(L, ldl, n, dmax, fail, sL);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  tol_rel = df_tol(tol_rel, split);
  for (int j0 = 0; j0 < n; j0 += CB) {
    const int bs = min(CB, n - j0);
    if ((e = diag_step(L, ldl, j0, bs, dmax, tol_rel, fail, sL, batch, split, n, (long long)n * CB, nullptr, 0, s)) !=
        cudaSuccess)
      return e;
    const int rem = n - j0 - bs;
    if (rem <= 0) break;
    if ((e = panel_step(L, ldl, j0, bs, rem, fail, sL, batch, split, n, (long long)n * CB, s)) != cudaSuccess)
      return e;
    e = trail_update(L, ldl, j0, bs, rem, batch, fail, sL, s, split, n, (long long)n * CB);
    if (e != cudaSuccess) return e;
  }
  note_launch();
  k_zero_upper<<<dim3((n + 127) / 128, n, batch), 128, 0, s>>>(L, ldl, n, sL);
  return cudaGetLastError();
}

}  // namespace isdf
