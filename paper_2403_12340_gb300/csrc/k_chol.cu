// Cholesky factorisation with optional diagonal pivoting, as one persistent
// cooperative kernel over all SMs.
//
// Used for C C^T (the ISDF least-squares normal matrix, pivoted: its rank
// drops below N_mu when there are more points than independent pairs) and
// for the two capacitance factors D = R R^T and I + R^T G R = U U^T (no
// pivoting; both are symmetric positive definite).
//
// Left-looking by columns: at step j the pivot p is the remaining row with
// the largest updated diagonal d[p]; column j of the factor is
//   L(i, j) = (W(i, p) - sum_{q<j} L(i, q) L(p, q)) / sqrt(d[p])
// for every remaining row i, then d[i] -= L(i, j)^2.  Rows are spread over
// the blocks (row i belongs to block i mod gridDim.x), one warp per row with
// lanes striding over q, so each step is one distributed matrix-vector
// product plus a grid-wide argmax.  FP64 on GB300 runs 7.9 GFLOP/s per SM,
// so the factorisation must use every SM; one grid barrier per column.
//
// The factor is kept row-major with rows in original order (Lr[i * n + q]),
// which makes the dot products coalesced.  Data written by other blocks is
// read with __ldcg (L2) so no stale L1 line is used after a barrier.
#include <cooperative_groups.h>

#include "common.cuh"
#include "kernels.h"

namespace isdf {

struct CholArgs {
  const double* W;
  long long ldw;
  int n;
  int pivot;
  double tol_rel;
  double* Lr;
  int* perm;
  int* rank;
  unsigned* status;
  double* d;
  double* part_val;
  int* part_idx;
  int* used;
  GridBarrier bar;
  uint64_t limit_ns;
};

__device__ __forceinline__ void argmax_merge(double& v, int& i, double v2, int i2) {
  // larger value wins; ties go to the lower index; NaN never wins
  if (v2 > v || (v2 == v && i2 < i) || (i < 0 && i2 >= 0)) {
    v = v2;
    i = i2;
  }
}

// Block-wide argmax of (val, idx) over threads; result valid in thread 0.
__device__ void block_argmax(double& v, int& i) {
  __shared__ double sv[32];
  __shared__ int si[32];
  for (int o = 16; o > 0; o >>= 1) {
    double v2 = __shfl_down_sync(0xffffffffu, v, o);
    int i2 = __shfl_down_sync(0xffffffffu, i, o);
    argmax_merge(v, i, v2, i2);
  }
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    sv[w] = v;
    si[w] = i;
  }
  __syncthreads();
  if (w == 0) {
    int nw = (blockDim.x + 31) >> 5;
    v = lane < nw ? sv[lane] : -1.0;
    i = lane < nw ? si[lane] : -1;
    for (int o = 16; o > 0; o >>= 1) {
      double v2 = __shfl_down_sync(0xffffffffu, v, o);
      int i2 = __shfl_down_sync(0xffffffffu, i, o);
      argmax_merge(v, i, v2, i2);
    }
  }
  __syncthreads();
}

// Local argmax of d over this block's remaining rows -> part_val/part_idx[buf][block].
// The partials are double-buffered by step parity: a block that has finished
// step j publishes for step j + 1 into the other buffer while slower blocks
// may still be reading the candidates of step j; none can reach step j + 2
// before every block has passed the barrier that ends step j.
__device__ void publish_local_max(const CholArgs& a, int buf) {
  double v = -1.0;
  int idx = -1;
  for (int i = blockIdx.x + gridDim.x * threadIdx.x; i < a.n; i += gridDim.x * blockDim.x) {
    if (!a.used[i]) argmax_merge(v, idx, __ldcg(&a.d[i]), i);
  }
  block_argmax(v, idx);
  if (threadIdx.x == 0) {
    a.part_val[buf * gridDim.x + blockIdx.x] = v;
    a.part_idx[buf * gridDim.x + blockIdx.x] = idx;
  }
}

// Every block reduces all partials (identical result in every block).
__device__ void global_max(const CholArgs& a, int buf, double& v, int& idx) {
  __shared__ double s_v;
  __shared__ int s_i;
  double bv = -1.0;
  int bi = -1;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
    argmax_merge(bv, bi, __ldcg(&a.part_val[buf * gridDim.x + b]), __ldcg(&a.part_idx[buf * gridDim.x + b]));
  block_argmax(bv, bi);
  if (threadIdx.x == 0) {
    s_v = bv;
    s_i = bi;
  }
  __syncthreads();
  v = s_v;
  idx = s_i;
}

__global__ void __launch_bounds__(256) k_cholesky(CholArgs a) {
  const int n = a.n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  // init: working diagonal, used flags (each block owns rows i = b mod G)
  for (int i = blockIdx.x + gridDim.x * threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    a.d[i] = a.W[i + a.ldw * (long long)i];
    a.used[i] = 0;
  }
  __syncthreads();
  publish_local_max(a, 0);
  if (!grid_sync(a.bar, a.status, a.limit_ns)) return;
  double dmax0;
  int p0;
  global_max(a, 0, dmax0, p0);
  const double thresh = a.tol_rel * dmax0;
  int rank = n;
  for (int j = 0; j < n; ++j) {
    double dp;
    int p;
    if (a.pivot) {
      if (j == 0) {
        dp = dmax0;
        p = p0;
      } else {
        global_max(a, j & 1, dp, p);
      }
    } else {
      p = j;
      dp = __ldcg(&a.d[j]);
    }
    if (!(dp > thresh) || p < 0) {  // also catches NaN
      rank = j;
      if (!a.pivot && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(a.status, ST_NOT_SPD);
      break;
    }
    const double ljj = sqrt(dp);
    const double inv = 1.0 / ljj;
    const double* Lp = a.Lr + (long long)p * n;
    // rows of this block: i = blockIdx.x + gridDim.x * t, one warp per row
    int t = warp;
    for (int i = blockIdx.x + gridDim.x * t; i < n; t += nwarps, i = blockIdx.x + gridDim.x * t) {
      double* Li = a.Lr + (long long)i * n;
      if (i == p) {
        if (lane == 0) {
          Li[j] = ljj;
          a.used[i] = 1;
        }
        continue;
      }
      if (a.used[i]) {
        if (lane == 0) Li[j] = 0.0;
        continue;
      }
      double acc = 0.0;
#pragma unroll 4
      for (int q = lane; q < j; q += 32) acc = fma(__ldcg(&Li[q]), __ldcg(&Lp[q]), acc);
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) {
        double wip = a.W[i + a.ldw * (long long)p];
        double l = (wip - acc) * inv;
        Li[j] = l;
        a.d[i] = __ldcg(&a.d[i]) - l * l;
      }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) a.perm[j] = p;
    __syncthreads();
    if (a.pivot) publish_local_max(a, (j + 1) & 1);
    if (!grid_sync(a.bar, a.status, a.limit_ns)) return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *a.rank = rank;
}

cudaError_t launch_cholesky(const double* W, long long ldw, int n, int pivot, double tol_rel,
                            double* Lr, int* perm, int* rank, unsigned* status, const CholWork& w,
                            int num_sms, uint64_t limit_ns, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cholesky, 256, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
  int blocks = num_sms;  // one block per SM: co-resident by construction
  if (blocks > w.max_blocks) blocks = w.max_blocks;  // partial arrays hold 2 * max_blocks
  if (blocks > n) blocks = n;
  if (blocks < 1) blocks = 1;
  e = cudaMemsetAsync(w.bar, 0, 2 * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  CholArgs a;
  a.W = W;
  a.ldw = ldw;
  a.n = n;
  a.pivot = pivot;
  a.tol_rel = tol_rel;
  a.Lr = Lr;
  a.perm = perm;
  a.rank = rank;
  a.status = status;
  a.d = w.d;
  a.part_val = w.part_val;
  a.part_idx = w.part_idx;
  a.used = w.used;
  a.bar = GridBarrier{w.bar, w.bar + 1};
  a.limit_ns = limit_ns;
  void* args[] = {&a};
  note_launch();
  return cudaLaunchCooperativeKernel((const void*)k_cholesky, dim3(blocks), dim3(256), args, 0, s);
}

// Diagnostic of the bounded grid barrier: every block enters grid_sync on a
// barrier whose arrival counter the caller preset past the grid size, so no
// block is the last to arrive and the generation never moves; each block
// gives up after limit_ns, sets ST_TIMEOUT and returns.
__global__ void k_wait_check(GridBarrier bar, unsigned* status, uint64_t limit_ns) {
  if (!grid_sync(bar, status, limit_ns)) return;
}

cudaError_t launch_wait_check(unsigned* bar, unsigned* status, uint64_t limit_ns, cudaStream_t s) {
  // counter 0x40404040, generation 0: no arrival count reaches gridDim - 1
  cudaError_t e = cudaMemsetAsync(bar, 0x40, sizeof(unsigned), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(bar + 1, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  GridBarrier b{bar, bar + 1};
  void* args[] = {&b, &status, &limit_ns};
  note_launch();
  return cudaLaunchCooperativeKernel((const void*)k_wait_check, dim3(2), dim3(32), args, 0, s);
}

}  // namespace isdf
