// Split-precision GEMM on the 5th-generation tensor cores (tcgen05).
//
// An FP64 operand x is represented by s BF16 slices, x ~ x0 + x1 + x2 with
// x0 = bf16(x), x1 = bf16(x - x0), x2 = bf16(x - x0 - x1) (s <= 3), stored
// K-major ("slice matrices": slice l of a R x K operand occupies rows
// [l Rp, l Rp + R) of a row-major (s Rp) x Kp BF16 array, zero padded).
// C = sum over slice pairs (i, j) with i + j < s of A_i B_j^T, accumulated in
// FP32 in tensor memory; dropping the pairs with i + j >= s costs about
// 2^-8s relative, so s = 3 gives FP32-grade products from six BF16 MMAs.
// Long K is split across thread blocks whose FP32 partial tiles are summed
// in FP64 (deterministically) afterwards.
//
// Kernel structure, one 128 x BN output tile per block (BN = 128):
//   warp 0  : TMA producer, s A-slice and s B-slice tiles (128 B rows,
//             128-byte swizzle) per 64-wide k chunk into a 2-4 stage ring;
//   warp 1  : allocates TMEM, issues tcgen05.mma (one thread), commits to
//             the ring's empty barriers and finally to the done barrier;
//   warps 2-5: epilogue, tcgen05.ld of the FP32 accumulator rows (TMEM lane
//             = tile row), FP64 conversion and the store.
// NACC = 2 runs two accumulators over two K ranges (the occupied and the
// unoccupied part of the orbital index) and multiplies them in the epilogue:
// the face-split Gram (Phi_v Phi_v,mu^T) .* (Phi_c Phi_c,mu^T) of the ISDF fit.
#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>

#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "../../include/isdf_smw.h"
#include "kernels.h"
#include "tc.cuh"

namespace isdf {

namespace {

constexpr int TC_BM = 128;
constexpr int TC_BK = 64;             // BF16 elements per 128-byte row
constexpr int TC_THREADS = 192;
constexpr int TC_SMEM_LIMIT = 227 * 1024;

__host__ __device__ inline int tc_stage_bytes(int s, int bn) { return s * (TC_BM + bn) * TC_BK * 2; }

__host__ __device__ inline int tc_stages(int s, int bn) {
  int per = tc_stage_bytes(s, bn);
  int st = (TC_SMEM_LIMIT - 2048) / per;
  return st > 4 ? 4 : st;
}

// Three BF16 slices of an FP32 value: a = bf16(x), b = bf16(x - a),
// c = bf16(x - a - b); the differences are exact in FP32, and a + b + c
// carries the 24 bits of x.  FP64 inputs are first rounded to FP32 with
// integer operations (no FP64 instructions on this path).
__device__ __forceinline__ void split3f(float x, __nv_bfloat16& a, __nv_bfloat16& b, __nv_bfloat16& c) {
  a = __float2bfloat16_rn(x);
  const float r = x - __bfloat162float(a);
  b = __float2bfloat16_rn(r);
  c = __float2bfloat16_rn(r - __bfloat162float(b));
}
__device__ __forceinline__ void split3(double x, __nv_bfloat16& a, __nv_bfloat16& b, __nv_bfloat16& c) {
  split3f(tc::d2f(x), a, b, c);
}
__device__ __forceinline__ void split3(float x, __nv_bfloat16& a, __nv_bfloat16& b, __nv_bfloat16& c) {
  split3f(x, a, b, c);
}

}  // namespace

// ------------------------------------------------------------- slicing

// 8 consecutive values -> 8 BF16 of each of the s slices, one 16-byte store
// per slice (dst must be 16-byte aligned).
template <class V>
__device__ __forceinline__ void store_slices8(const V (&v)[8], __nv_bfloat16* dst, long long sstr, int s) {
  __align__(16) __nv_bfloat16 x0[8], x1[8], x2[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) split3(v[q], x0[q], x1[q], x2[q]);
  *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(x0);
  if (s > 1) *reinterpret_cast<uint4*>(dst + sstr) = *reinterpret_cast<const uint4*>(x1);
  if (s > 2) *reinterpret_cast<uint4*>(dst + 2 * sstr) = *reinterpret_cast<const uint4*>(x2);
}

// Column-major FP64 source (element (row, col) at src[row + lds col]) ->
// slices dst[(l Rp + row) Kp + kmap(col)], kmap(col) = col for col < kv,
// col - kv + kvp otherwise (kv = kvp = 0: identity).  64 x 64 tiles through
// shared memory: coalesced FP64 loads down the columns, 16-byte slice stores
// along the rows where the destination is 16-byte aligned (Kp % 8 == 0),
// element stores elsewhere.
__global__ void __launch_bounds__(256) k_slice_cm(const double* __restrict__ src, long long lds, int R, int C, int kv,
                                                  int kvp, __nv_bfloat16* __restrict__ dst, int Rp, int Kp, int s,
                                                  long long sstride, long long dstride) {
  __shared__ double t[64][65];
  src += sstride * blockIdx.z;
  dst += dstride * blockIdx.z;
  const int r0 = blockIdx.x * 64, c0 = blockIdx.y * 64;
  for (int idx = threadIdx.x; idx < 64 * 64; idx += 256) {
    int rr = idx & 63, cc = idx >> 6;
    int r = r0 + rr, c = c0 + cc;
    t[cc][rr] = (r < R && c < C) ? src[r + lds * (long long)c] : 0.0;
  }
  __syncthreads();
  const long long sstr = (long long)Rp * Kp;
  for (int idx = threadIdx.x; idx < 64 * 8; idx += 256) {
    const int rr = idx >> 3, ch = idx & 7;
    const int r = r0 + rr, cb = c0 + ch * 8;
    if (r >= R || cb >= C) continue;
    double v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = t[ch * 8 + q][rr];
    // a 16-byte store needs the whole chunk on one side of kv and, past kv,
    // a shift kvp - kv that keeps the destination 8-aligned
    const bool whole = cb + 8 <= C && (cb + 8 <= kv || (cb >= kv && ((kvp - kv) & 7) == 0));
    if (whole) {
      const int kc = (cb < kv) ? cb : cb - kv + kvp;
      store_slices8(v, dst + (long long)r * Kp + kc, sstr, s);
    } else {
      for (int q = 0; q < 8 && cb + q < C; ++q) {
        const int c = cb + q;
        const int kc = (c < kv) ? c : c - kv + kvp;
        __nv_bfloat16 a, b, d;
        split3(v[q], a, b, d);
        const long long base = (long long)r * Kp + kc;
        dst[base] = a;
        if (s > 1) dst[base + sstr] = b;
        if (s > 2) dst[base + 2 * sstr] = d;
      }
    }
  }
}

// Row-major FP64 source (element (row, k) at src[k + lds row]) -> slices;
// eight k per thread, 16-byte slice stores.
__global__ void k_slice_rm(const double* __restrict__ src, long long lds, int R, int K,
                           __nv_bfloat16* __restrict__ dst, int Rp, int Kp, int s, long long sstride,
                           long long dstride) {
  src += sstride * blockIdx.z;
  dst += dstride * blockIdx.z;
  const int row = blockIdx.y;
  const long long sstr = (long long)Rp * Kp;
  const double* in = src + lds * (long long)row;
  for (int k8 = (blockIdx.x * blockDim.x + threadIdx.x) * 8; k8 < K; k8 += gridDim.x * blockDim.x * 8) {
    double v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = (k8 + q < K) ? in[k8 + q] : 0.0;
    store_slices8(v, dst + (long long)row * Kp + k8, sstr, s);
  }
}

cudaError_t launch_slice_colmajor(const double* src, long long lds, int R, int C, int kv, int kvp,
                                  __nv_bfloat16* dst, int Rp, int Kp, int s, cudaStream_t st, int batch,
                                  long long sstride, long long dstride) {
  if (R <= 0 || C <= 0 || batch <= 0) return cudaSuccess;
  if (Kp % 8 || batch > 65535 || (dstride % 8)) return cudaErrorInvalidValue;
  dim3 grid((R + 63) / 64, (C + 63) / 64, batch);
  KernelTimer kt(KF_SLICE, st, (double)R * C * (8.0 + 2.0 * s) * batch);
  note_launch();
  k_slice_cm<<<grid, 256, 0, st>>>(src, lds, R, C, kv, kvp, dst, Rp, Kp, s, sstride, dstride);
  return cudaGetLastError();
}

cudaError_t launch_slice_rowmajor(const double* src, long long lds, int R, int K, __nv_bfloat16* dst, int Rp,
                                  int Kp, int s, cudaStream_t st, int batch, long long sstride, long long dstride) {
  if (R <= 0 || K <= 0 || batch <= 0) return cudaSuccess;
  if (Kp % 8 || Kp < (K + 7) / 8 * 8 || R > 65535 || batch > 65535 || (dstride % 8)) return cudaErrorInvalidValue;
  int bx = (K + 2047) / 2048;
  if (bx > 64) bx = 64;
  dim3 grid(bx, R, batch);
  KernelTimer kt(KF_SLICE, st, (double)R * K * (8.0 + 2.0 * s) * batch);
  note_launch();
  k_slice_rm<<<grid, 256, 0, st>>>(src, lds, R, K, dst, Rp, Kp, s, sstride, dstride);
  return cudaGetLastError();
}

// Slices of the pair operand of the polarizability at the points:
// S(a, i n_c + j) = phimu(a, i) phimu(a, n_v + j) sw[i n_c + j], a < r
// (the columns of C, Eq. MatrixExpressionISDF, scaled by sqrt(-2 Omega^-1)),
// and zero in the padding (rows r..Rp, columns K..Kp), so the destination
// needs no clearing.  A block converts PS_ROWS rows of phimu to FP32 into
// shared memory once, then each thread writes eight consecutive pairs of
// all PS_ROWS rows: the weights (FP32, the same rounding as before) are read
// once for PS_ROWS rows and every slice store is 16 bytes.  The kernel is
// bound by its writes, 2 s bytes per element.
constexpr int PS_ROWS = 4;

__global__ void __launch_bounds__(256) k_pair_slices(const double* __restrict__ phimu, long long ldp, int r, int n_v,
                                                     int n_c, const float* __restrict__ swf,
                                                     __nv_bfloat16* __restrict__ dst, int Rp, int Kp, int s,
                                                     long long dstride) {
  extern __shared__ float ps_rows[];  // PS_ROWS x n_e
  const int n_e = n_v + n_c, K = n_v * n_c;
  const int a0 = blockIdx.y * PS_ROWS;
  swf += (long long)K * blockIdx.z;
  dst += dstride * blockIdx.z;
  for (int idx = threadIdx.x; idx < PS_ROWS * n_e; idx += blockDim.x) {
    const int q = idx / n_e, e = idx - q * n_e;
    ps_rows[idx] = (a0 + q < r) ? tc::d2f(phimu[(a0 + q) + ldp * (long long)e]) : 0.f;
  }
  __syncthreads();
  const long long sstr = (long long)Rp * Kp;
  for (int k8 = (blockIdx.x * blockDim.x + threadIdx.x) * 8; k8 < Kp; k8 += gridDim.x * blockDim.x * 8) {
    float w[8];
    int iv[8], jc[8];
    int i = k8 / n_c, j = k8 - i * n_c;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const bool in = k8 + q < K;
      w[q] = in ? swf[k8 + q] : 0.f;
      iv[q] = in ? i : 0;
      jc[q] = in ? j : 0;
      if (++j == n_c) {
        j = 0;
        ++i;
      }
    }
#pragma unroll
    for (int q = 0; q < PS_ROWS; ++q) {
      const float* row = ps_rows + q * n_e;
      float v[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) v[e] = row[iv[e]] * row[n_v + jc[e]] * w[e];
      store_slices8(v, dst + (long long)(a0 + q) * Kp + k8, sstr, s);
    }
  }
}

// Slices of the unscaled pair operand, transposed: rows are the pairs
// p = i n_c + j, the K index the r points, value phimu(a, i) phimu(a, n_v + j);
// eight points per thread, 16-byte slice stores.
__global__ void k_pair_slices_t(const double* __restrict__ phimu, long long ldp, int r, int n_v, int n_c,
                                __nv_bfloat16* __restrict__ dst, int Pp, int Kp, int s) {
  const long long p = blockIdx.y * (long long)gridDim.x + blockIdx.x;
  if (p >= (long long)n_v * n_c) return;
  const int i = (int)(p / n_c), j = (int)(p - (long long)i * n_c);
  const double* pv = phimu + ldp * (long long)i;
  const double* pc = phimu + ldp * (long long)(n_v + j);
  const long long sstr = (long long)Pp * Kp;
  for (int a8 = threadIdx.x * 8; a8 < r; a8 += blockDim.x * 8) {
    float v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = (a8 + q < r) ? tc::d2f(pv[a8 + q]) * tc::d2f(pc[a8 + q]) : 0.f;
    store_slices8(v, dst + p * Kp + a8, sstr, s);
  }
}

cudaError_t launch_pair_slices_t(const double* phimu, long long ldp, int r, int n_v, int n_c, __nv_bfloat16* dst,
                                 int Pp, int Kp, int s, cudaStream_t st) {
  const long long np = (long long)n_v * n_c;
  if (r <= 0 || np <= 0) return cudaSuccess;
  if (Kp % 8 || Kp < r) return cudaErrorInvalidValue;
  const unsigned gx = (unsigned)std::min<long long>(np, 65535);
  dim3 grid(gx, (unsigned)((np + gx - 1) / gx));
  KernelTimer kt(KF_SLICE, st, (double)r * (n_v + n_c) * 8.0 + (double)np * r * 2.0 * s);
  note_launch();
  k_pair_slices_t<<<grid, 128, 0, st>>>(phimu, ldp, r, n_v, n_c, dst, Pp, Kp, s);
  return cudaGetLastError();
}

cudaError_t launch_pair_slices(const double* phimu, long long ldp, int r, int n_v, int n_c, const float* swf,
                               __nv_bfloat16* dst, int Rp, int Kp, int s, cudaStream_t st, int batch,
                               long long dstride) {
  if (r <= 0 || batch <= 0) return cudaSuccess;
  const int K = n_v * n_c, n_e = n_v + n_c;
  if (batch > 65535 || Rp % PS_ROWS || Rp < r || Rp / PS_ROWS > 65535 || Kp % 8 || Kp < K || (dstride % 8))
    return cudaErrorInvalidValue;
  const size_t smem = (size_t)PS_ROWS * n_e * sizeof(float);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  static size_t smem_set = 48 * 1024;
  if (smem > smem_set) {
    cudaError_t e = cudaFuncSetAttribute(k_pair_slices, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    smem_set = 200 * 1024;
  }
  const int bx = std::min((Kp + 2047) / 2048, 8);
  dim3 grid(bx, Rp / PS_ROWS, batch);
  KernelTimer kt(KF_SLICE, st, ((double)r * n_e * 8.0 + (double)K * 4.0 * (Rp / PS_ROWS) +
                                (double)Rp * Kp * 2.0 * s) * batch);
  note_launch();
  k_pair_slices<<<grid, 256, smem, st>>>(phimu, ldp, r, n_v, n_c, swf, dst, Rp, Kp, s, dstride);
  return cudaGetLastError();
}

// ------------------------------------------------------------ the GEMM

struct TcArgs {
  int M, N;
  int a_rows_pad, b_rows_pad;  // slice stride (rows) of the A / B slice matrices
  int s;                       // slices per operand (1..3)
  int k_iters;                 // Kp / 64
  int k_per_split;             // k chunks per blockIdx.z
  int kv_iters;                // NACC == 2: chunks of the first accumulator
  int lower_only;              // M == N; only tiles with n-tile <= m-tile
  int tri_b;                   // B(n, k) == 0 for k > n: skip chunks beyond the tile's last n
  int group;                   // NACC == 1: 64-wide K chunks per FP32 accumulation run (0: the whole unit)
  int tiles_m, tiles_n;        // tiles along M and N
  int count;                   // problems of the batch
  int splits;                  // K splits per problem (units: problem, split, tile)
  int tma3;                    // the maps are 3-D (chunk, row, slab): one load brings every slice
  int a_brows, b_brows;        // rows between the slice stacks of consecutive problems (0: shared)
  long long c_bstride;         // elements between the C of consecutive problems
  double alpha, beta;
  double* C;
  long long ldc;
  double* partial;             // raw FP64 partial tiles [z][M N] (column-major M x N)
  __nv_bfloat16* zs;           // EPI_HAD_SLICES / EPI_SCALE_SLICES output slices (row-major)
  int zs_rows_pad, zs_kp;
  long long zs_bstride;        // elements between the output slices of consecutive problems
  const float* colscale;       // EPI_SCALE_SLICES: column n of problem b scaled by colscale[b cs_bstride + n]
  long long cs_bstride;
  __nv_bfloat16* zt;           // EPI_F64_SLICES2: slices of C transposed, element (n, m) at zt[n zt_kp + m]
  int zt_rows_pad, zt_kp;
  unsigned* status;
};

enum { EPI_F64 = 0, EPI_HAD_F64 = 1, EPI_HAD_SLICES = 2, EPI_SCALE_SLICES = 3, EPI_F64_SLICES2 = 4 };

// One work unit: a 128 x BN output tile of one problem over one K range.
struct TcUnit {
  int mt, nt, m0, n0, bidx, split, kb, ke;
};

__device__ __forceinline__ TcUnit tc_unit(const TcArgs& a, long long u, int tiles, int bn) {
  TcUnit w;
  const long long per_b = (long long)a.splits * tiles;
  w.bidx = (int)(u / per_b);
  const long long rem = u - (long long)w.bidx * per_b;
  w.split = (int)(rem / tiles);
  const int tile = (int)(rem - (long long)w.split * tiles);
  if (a.lower_only) {
    lower_tile(tile, w.mt, w.nt);
  } else {
    w.mt = tile / a.tiles_n;  // n fastest: consecutive units share the A tile (L2 reuse)
    w.nt = tile - w.mt * a.tiles_n;
    // under tri_b a tile's K range grows with nt; rotating nt by the row
    // spreads long and short tiles over the persistent blocks (at isdf48
    // the busiest block then does 5 % more than the mean instead of 25 %)
    if (a.tri_b) w.nt = (w.nt + w.mt) % a.tiles_n;
  }
  w.m0 = w.mt * TC_BM;
  w.n0 = w.nt * bn;
  w.kb = w.split * a.k_per_split;
  w.ke = min(a.k_iters, w.kb + a.k_per_split);
  if (a.tri_b) w.ke = min(w.ke, (w.n0 + bn + TC_BK - 1) / TC_BK);
  if (w.ke < w.kb) w.ke = w.kb;
  return w;
}

// Persistent: block b computes units b, b + gridDim.x, ...; the stage ring
// runs on across units, and the accumulator alternates between two TMEM
// buffers so that the epilogue of one unit overlaps the MMAs of the next.
template <int BN, int NACC, int EPI>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap tma, const __grid_constant__ CUtensorMap tmb, TcArgs a) {
  extern __shared__ __align__(1024) uint8_t tc_smem_raw[];
  // 1024-byte aligned ring of stages, then the barriers
  uint8_t* smem = (uint8_t*)(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
  const int S = tc_stages(a.s, BN);
  const int stage_bytes = tc_stage_bytes(a.s, BN);
  uint64_t* full = (uint64_t*)(smem + S * stage_bytes);
  uint64_t* empty = full + 4;
  uint64_t* tfull = empty + 4;   // accumulator buffer b holds a finished unit (MMA -> epilogue)
  uint64_t* tempty = tfull + 2;  // accumulator buffer b has been read (epilogue -> MMA), 4 warps
  uint32_t* tmem_slot = (uint32_t*)(tempty + 2);
  __shared__ int s_abort;
  constexpr uint32_t ACC_COLS = NACC * BN;
  // Grouped accumulation (NACC == 1, a.group > 0): each unit's K range runs
  // as groups of a.group chunks, each summed in FP32 in one accumulator
  // buffer, and the epilogue adds every group into a double-float running
  // sum (hi, lo) kept in two more TMEM column blocks; the FP32 rounding then
  // builds up over a.group * 64 terms at most instead of the whole range.
  const bool grouped = NACC == 1 && a.group > 0;
  const uint32_t tcols = grouped ? 2 * ACC_COLS + 2 * BN : 2 * ACC_COLS;  // 512 or 256 for BN 128 / 64
  const uint32_t df_hi = 2 * ACC_COLS, df_lo = 2 * ACC_COLS + BN;       // column offsets of the running sum

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tiles = a.lower_only ? a.tiles_m * (a.tiles_m + 1) / 2 : a.tiles_m * a.tiles_n;
  const long long units = (long long)a.count * a.splits * tiles;

  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int i = 0; i < S; ++i) {
      tc::mbar_init(&full[i], 1);
      tc::mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(&tfull[i], 1);
      tc::mbar_init(&tempty[i], 4);
    }
    tc::fence_mbar_init();
  }
  if (warp == 1) tc::tmem_alloc(tmem_slot, tcols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer
    tc::prefetch_tmap(&tma);
    tc::prefetch_tmap(&tmb);
    const uint32_t bytes = (uint32_t)stage_bytes;
    uint32_t g = 0;  // stage-ring position, continuous across units
    for (long long u = blockIdx.x; u < units && !s_abort; u += gridDim.x) {
      const TcUnit w = tc_unit(a, u, tiles, BN);
      const int a_row0 = w.bidx * a.a_brows + w.m0, b_row0 = w.bidx * a.b_brows + w.n0;
      for (int kc = w.kb; kc < w.ke; ++kc, ++g) {
        const int st = (int)(g % (uint32_t)S);
        const uint32_t ph = (g / (uint32_t)S) & 1u;
        if (!tc::mbar_wait(&empty[st], ph ^ 1u, a.status)) {
          s_abort = 1;
          break;
        }
        tc::mbar_expect_tx(&full[st], bytes);
        uint8_t* sa = smem + st * stage_bytes;
        uint8_t* sb = sa + a.s * TC_BM * TC_BK * 2;
        const int kx = kc * TC_BK;
        if (a.tma3) {  // the s slices of each operand in one copy each (slabs of rows_pad rows)
          tc::tma_load_3d(sa, &tma, &full[st], kx, w.m0, w.bidx * (a.a_brows / a.a_rows_pad));
          tc::tma_load_3d(sb, &tmb, &full[st], kx, w.n0, w.bidx * (a.b_brows / a.b_rows_pad));
        } else {
          for (int l = 0; l < a.s; ++l) {
            tc::tma_load_2d(sa + l * TC_BM * TC_BK * 2, &tma, &full[st], kx, a_row0 + l * a.a_rows_pad);
            tc::tma_load_2d(sb + l * BN * TC_BK * 2, &tmb, &full[st], kx, b_row0 + l * a.b_rows_pad);
          }
        }
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    constexpr uint32_t idesc = tc::idesc_bf16_f32(TC_BM, BN);
    uint32_t g = 0;
    uint32_t gi = 0;  // accumulation groups issued by this block (one per unit unless grouped)
    bool stop = false;
    for (long long u = blockIdx.x; u < units && !s_abort && !stop; u += gridDim.x) {
      const TcUnit w = tc_unit(a, u, tiles, BN);
      const int ng = (grouped && w.ke > w.kb) ? (w.ke - w.kb + a.group - 1) / a.group : 1;
      int kc = w.kb;
      for (int gr = 0; gr < ng; ++gr, ++gi) {
      const int buf = (int)(gi & 1u);
      // the epilogue has read this buffer's previous group (two groups ago)
      if (!tc::mbar_wait(&tempty[buf], ((gi >> 1) & 1u) ^ 1u, a.status)) {
        s_abort = 1;
        stop = true;
        break;
      }
      tc::fence_after_sync();
      const uint32_t dbase = tmem + (uint32_t)buf * ACC_COLS;
      bool first[2] = {true, true};
      bool ok = true;
      const int kg0 = kc;
      const int kend = grouped ? min(w.ke, kc + a.group) : w.ke;
      for (; kc < kend; ++kc, ++g) {
        const int st = (int)(g % (uint32_t)S);
        const uint32_t ph = (g / (uint32_t)S) & 1u;
        if (!tc::mbar_wait(&full[st], ph, a.status)) {
          ok = false;
          break;
        }
        tc::fence_after_sync();
        const int acc = (NACC == 2 && kc >= a.kv_iters) ? 1 : 0;
        const uint32_t d = dbase + (uint32_t)(acc * BN);
        const uint32_t sa = tc::smem_u32(smem + st * stage_bytes);
        const uint32_t sb = sa + (uint32_t)(a.s * TC_BM * TC_BK * 2);
#pragma unroll
        for (int kk = 0; kk < TC_BK / 16; ++kk) {
          for (int i = 0; i < a.s; ++i) {
            for (int j = 0; i + j < a.s; ++j) {
              const uint64_t ad = tc::desc_kmajor_sw128(sa + (uint32_t)(i * TC_BM * TC_BK * 2 + kk * 32));
              const uint64_t bd = tc::desc_kmajor_sw128(sb + (uint32_t)(j * BN * TC_BK * 2 + kk * 32));
              tc::mma_bf16(d, ad, bd, idesc, first[acc] ? 0u : 1u);
              first[acc] = false;
            }
          }
        }
        tc::mma_commit(&empty[st]);  // the stage is free once these MMAs have read it
      }
      if (!ok) {
        s_abort = 1;
        stop = true;
        break;
      }
      if (kend > kg0) {
        tc::mma_commit(&tfull[buf]);
      } else {
        tc::mbar_arrive(&tfull[buf]);
      }
      }
    }
  } else if (warp >= 2) {
    // ---------------- epilogue: thread <-> tile row (TMEM lane)
    const int q = warp & 3;  // TMEM lane quarter this warp may access
    const int row = q * 32 + lane;
    uint32_t gi = 0;  // accumulation groups consumed, in the MMA warp's order
    bool stop = false;
    for (long long u = blockIdx.x; u < units && !stop; u += gridDim.x) {
      const TcUnit w = tc_unit(a, u, tiles, BN);
      const int ng = (grouped && w.ke > w.kb) ? (w.ke - w.kb + a.group - 1) / a.group : 1;
      for (int gr = 0; gr < ng; ++gr, ++gi) {
      const int buf = (int)(gi & 1u);
      const bool ok = tc::mbar_wait(&tfull[buf], (gi >> 1) & 1u, a.status);
      tc::fence_after_sync();
      if (!ok || s_abort) {
        stop = true;
        break;
      }
      const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16);
      const uint32_t lane_addr = lane_base + (uint32_t)buf * ACC_COLS;
      if (grouped && gr + 1 < ng) {
        // not the unit's last group: fold it into the double-float running sum
        for (int c = 0; c < BN; c += 16) {
          float v[16], hi[16], lo[16];
          tc::tmem_ld16(lane_addr + (uint32_t)c, v);
          if (gr == 0) {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              hi[i] = v[i];
              lo[i] = 0.f;
            }
          } else {
            tc::tmem_ld16(lane_base + df_hi + (uint32_t)c, hi);
            tc::tmem_ld16(lane_base + df_lo + (uint32_t)c, lo);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const float t = __fadd_rn(hi[i], v[i]);
              const float bv = __fsub_rn(t, hi[i]);
              const float err = __fadd_rn(__fsub_rn(hi[i], __fsub_rn(t, bv)), __fsub_rn(v[i], bv));
              const float l = __fadd_rn(lo[i], err);
              hi[i] = __fadd_rn(t, l);
              lo[i] = __fsub_rn(l, __fsub_rn(hi[i], t));
            }
          }
          tc::tmem_st16(lane_base + df_hi + (uint32_t)c, hi);
          tc::tmem_st16(lane_base + df_lo + (uint32_t)c, lo);
        }
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&tempty[buf]);
        continue;
      }
      const bool with_sum = grouped && gr > 0;  // the unit's result is the running sum plus this group
      const int m = w.m0 + row;
      const bool have = w.ke > w.kb;
      const bool have1 = NACC == 2 && have && w.ke > a.kv_iters;
      const bool have0 = have && (NACC == 1 || w.kb < a.kv_iters);
      double* Cb = a.C + a.c_bstride * w.bidx;
      for (int c = 0; c < BN; c += 16) {
        float v0[16], v1[16], w0[16];
        if (have0) tc::tmem_ld16(lane_addr + (uint32_t)c, v0);
        else
          for (int i = 0; i < 16; ++i) v0[i] = 0.f;
#pragma unroll
        for (int i = 0; i < 16; ++i) w0[i] = 0.f;
        if (with_sum) {
          // (hi, lo) + v0 -> (v0, w0): the value to 48 bits, high part in v0
          float hi[16], lo[16];
          tc::tmem_ld16(lane_base + df_hi + (uint32_t)c, hi);
          tc::tmem_ld16(lane_base + df_lo + (uint32_t)c, lo);
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const float t = __fadd_rn(hi[i], v0[i]);
            const float bv = __fsub_rn(t, hi[i]);
            const float err = __fadd_rn(__fsub_rn(hi[i], __fsub_rn(t, bv)), __fsub_rn(v0[i], bv));
            const float l = __fadd_rn(lo[i], err);
            v0[i] = __fadd_rn(t, l);
            w0[i] = __fsub_rn(l, __fsub_rn(v0[i], t));
          }
        }
        if (NACC == 2) {
          if (have1) tc::tmem_ld16(lane_addr + (uint32_t)(BN + c), v1);
          else
            for (int i = 0; i < 16; ++i) v1[i] = 0.f;
        }
        if (m >= a.M) continue;
        if (EPI == EPI_F64_SLICES2) {
          // C in FP64 (alpha 1, beta 0), and its BF16 slices twice: row-major
          // (m, n) into zs and transposed (n, m) into zt
          const long long sstr = (long long)a.zs_rows_pad * a.zs_kp, tstr = (long long)a.zt_rows_pad * a.zt_kp;
          const bool whole = w.n0 + c + 16 <= a.N;
          if (whole) {
            __nv_bfloat16* dst = a.zs + (long long)m * a.zs_kp + w.n0 + c;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              float v[8];
#pragma unroll
              for (int e = 0; e < 8; ++e) v[e] = v0[8 * h + e];
              store_slices8(v, dst + 8 * h, sstr, a.s);
            }
          }
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int n = w.n0 + c + i;
            if (n >= a.N) break;
            Cb[m + a.ldc * n] = with_sum ? tc::f2d(v0[i]) + tc::f2d(w0[i]) : tc::f2d(v0[i]);
            __nv_bfloat16 x0, x1, x2;
            split3f(v0[i], x0, x1, x2);
            if (!whole) {
              const long long base = (long long)m * a.zs_kp + n;
              a.zs[base] = x0;
              if (a.s > 1) a.zs[base + sstr] = x1;
              if (a.s > 2) a.zs[base + 2 * sstr] = x2;
            }
            const long long tb = (long long)n * a.zt_kp + m;
            a.zt[tb] = x0;
            if (a.s > 1) a.zt[tb + tstr] = x1;
            if (a.s > 2) a.zt[tb + 2 * tstr] = x2;
          }
          continue;
        }
        const float* cs = (EPI == EPI_SCALE_SLICES) ? a.colscale + a.cs_bstride * w.bidx : nullptr;
        if ((EPI == EPI_HAD_SLICES || EPI == EPI_SCALE_SLICES) && w.n0 + c + 16 <= a.N) {
          // whole 16-column chunk: two 16-byte stores per slice
          const long long sstr = (long long)a.zs_rows_pad * a.zs_kp;
          __nv_bfloat16* dst = a.zs + a.zs_bstride * w.bidx + (long long)m * a.zs_kp + w.n0 + c;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            float v[8];
#pragma unroll
            for (int e = 0; e < 8; ++e)
              v[e] = (EPI == EPI_SCALE_SLICES) ? v0[8 * h + e] * cs[w.n0 + c + 8 * h + e] : v0[8 * h + e] * v1[8 * h + e];
            store_slices8(v, dst + 8 * h, sstr, a.s);
          }
          continue;
        }
        // beta C: the chunk's 16 loads issued together, ahead of the stores
        // (one memory round trip per chunk instead of one per element)
        double cin[16];
        const bool rd = (EPI == EPI_F64 || EPI == EPI_HAD_F64) && !a.partial && a.beta != 0.0;
        if (rd) {
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int n = w.n0 + c + i;
            cin[i] = (n < a.N && !(a.lower_only && n > m)) ? Cb[m + a.ldc * n] : 0.0;
          }
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int n = w.n0 + c + i;
          if (n >= a.N) break;
          const float vf = (EPI == EPI_SCALE_SLICES) ? v0[i] * cs[n] : ((NACC == 2) ? v0[i] * v1[i] : v0[i]);
          if (EPI == EPI_HAD_SLICES || EPI == EPI_SCALE_SLICES) {
            __nv_bfloat16 x0, x1, x2;
            split3f(vf, x0, x1, x2);
            long long base = a.zs_bstride * w.bidx + (long long)m * a.zs_kp + n;
            long long sstr = (long long)a.zs_rows_pad * a.zs_kp;
            a.zs[base] = x0;
            if (a.s > 1) a.zs[base + sstr] = x1;
            if (a.s > 2) a.zs[base + 2 * sstr] = x2;
          } else if (a.partial) {
            a.partial[((long long)w.bidx * a.splits + w.split) * a.M * a.N + m + (long long)a.M * n] =
                with_sum ? tc::f2d(vf) + tc::f2d(w0[i]) : tc::f2d(vf);
          } else {
            // lower-only: the lower triangle, mirrored (an exactly symmetric C;
            // beta reads only the lower triangle of C)
            if (a.lower_only && n > m) break;
            // alpha = 1, beta = 0 and no running sum (the common case) need no FP64 arithmetic
            const double vd = with_sum ? tc::f2d(vf) + tc::f2d(w0[i]) : tc::f2d(vf);
            double o = (a.alpha == 1.0) ? vd : a.alpha * vd;
            if (rd) o += a.beta * cin[i];
            Cb[m + a.ldc * n] = o;
            if (a.lower_only && n < m) Cb[n + a.ldc * m] = o;
          }
        }
      }
      // this warp has read its lanes of the buffer: hand it back to the MMA warp
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&tempty[buf]);
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 1) tc::tmem_dealloc(tmem, tcols);
}

// ------------------------------------------------------------ host side

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

// 2-D map over a row-major BF16 array (rows x kp), box 64 x box_rows, 128B swizzle.
static cudaError_t make_map(CUtensorMap* m, const __nv_bfloat16* base, int kp, long long rows, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  if (((uintptr_t)base & 15) || (kp % 8)) return cudaErrorInvalidValue;
  cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)kp * 2};
  cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// 3-D map over the same array seen as slabs of rows_pad rows (a slice of a
// stack, or a member of a batch): box 64 x box_rows x s, 128B swizzle.
static cudaError_t make_map3(CUtensorMap* m, const __nv_bfloat16* base, int kp, int rows_pad, long long slabs,
                             int box_rows, int s) {
  auto fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  if (((uintptr_t)base & 15) || (kp % 8)) return cudaErrorInvalidValue;
  cuuint64_t dims[3] = {(cuuint64_t)kp, (cuuint64_t)rows_pad, (cuuint64_t)slabs};
  cuuint64_t strides[2] = {(cuuint64_t)kp * 2, (cuuint64_t)kp * 2 * (cuuint64_t)rows_pad};
  cuuint32_t box[3] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows, (cuuint32_t)s};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int BN, int NACC, int EPI>
static cudaError_t tc_launch(const TcOperand& A, const TcOperand& B, TcArgs a, int splits, int batch,
                             double mma_flops, cudaStream_t st) {
  CUtensorMap ma, mb;
  const long long arows = (long long)A.rows_pad * a.s + (long long)a.a_brows * (batch - 1);
  const long long brows = (long long)B.rows_pad * a.s + (long long)a.b_brows * (batch - 1);
  cudaError_t e;
  // one 3-D copy per operand and stage when the stacks are whole slabs of
  // rows_pad rows and every tile lies inside one slab
  a.tma3 = A.rows_pad % TC_BM == 0 && B.rows_pad % BN == 0 && a.a_brows % A.rows_pad == 0 &&
           a.b_brows % B.rows_pad == 0;
  if (a.tma3) {
    e = make_map3(&ma, A.p, A.kp, A.rows_pad, arows / A.rows_pad, TC_BM, a.s);
    if (e == cudaSuccess) e = make_map3(&mb, B.p, B.kp, B.rows_pad, brows / B.rows_pad, BN, a.s);
    if (e != cudaSuccess) return e;
  } else {
    e = make_map(&ma, A.p, A.kp, arows, TC_BM);
    if (e != cudaSuccess) return e;
    e = make_map(&mb, B.p, B.kp, brows, BN);
    if (e != cudaSuccess) return e;
  }
  const int smem = tc_stages(a.s, BN) * tc_stage_bytes(a.s, BN) + 1024 + 256;
  // once per kernel (host threads of a batch may arrive together: setting it twice is harmless,
  // and a thread that reads true finds it set)
  static std::atomic<bool> configured{false};
  if (!configured.load(std::memory_order_acquire)) {
    e = cudaFuncSetAttribute(k_tc_gemm<BN, NACC, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             TC_SMEM_LIMIT - 2048);  // leaves room for the static shared variables
    if (e != cudaSuccess) return e;
    configured.store(true, std::memory_order_release);
  }
  if (smem > TC_SMEM_LIMIT - 2048) return cudaErrorInvalidValue;
  const int tm = (a.M + TC_BM - 1) / TC_BM, tn = (a.N + BN - 1) / BN;
  a.group = NACC == 1 ? tl_tc_group : 0;
  a.tiles_m = tm;
  a.tiles_n = tn;
  a.splits = splits;
  a.count = batch;
  const long long tiles = a.lower_only ? (long long)tm * (tm + 1) / 2 : (long long)tm * tn;
  const long long units = tiles * splits * batch;
  static std::atomic<int> sms_cache{0};
  int sms = sms_cache.load(std::memory_order_relaxed);
  if (!sms) {
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    sms_cache.store(sms, std::memory_order_relaxed);
  }
  // one block per SM (the stage ring takes most of the shared memory), each looping over units
  const int avail = std::max(1, sms - std::max(0, tl_tc_sm_reserve));
  dim3 grid((unsigned)std::min<long long>(units, avail));
  KernelTimer kt(KF_TC_GEMM, st, mma_flops);
  note_launch();
  k_tc_gemm<BN, NACC, EPI><<<grid, TC_THREADS, smem, st>>>(ma, mb, a);
  return cudaGetLastError();
}

static void split_k(int k_iters, int tiles, int num_sms, int max_split, int& splits, int& per) {
  int want = (2 * num_sms + tiles - 1) / tiles;
  const int accuracy = (k_iters + kTcMaxChunksPerSplit - 1) / kTcMaxChunksPerSplit;
  if (want < accuracy) want = accuracy;
  if (want > max_split) want = max_split;
  if (want > k_iters) want = k_iters;
  if (want < 1) want = 1;
  per = (k_iters + want - 1) / want;
  splits = (k_iters + per - 1) / per;
}

thread_local int tl_tc_sm_reserve = 0;
thread_local int tl_tc_group = kTcGroupChunks;

// ------------------------------------------------------------ tile autotuner
//
// The split-K count and the tile width of an EPI_F64 GEMM come from a
// heuristic (two units per SM, the accumulation-length minimum, 128-wide
// tiles).  With the autotuner on, the first call of each shape instead times
// the candidates -- the heuristic split, twice and half of it (within the
// accumulation minimum and the caller's partial buffer), each with 128- and
// 64-wide tiles (a 64-wide tile leaves room for three pipeline stages
// instead of two; lower-only SYRKs keep square tiles) -- on the call's own
// operands and output, and keeps the fastest for every later call of that
// shape, including calls recorded into a CUDA graph.  Calls that accumulate
// into C (beta != 0) keep the heuristic, because a timed candidate would
// change C.
struct TuneKey {
  int M, N, kp, s, lower, tri, count, max_split;
  bool operator<(const TuneKey& o) const {
    return std::tie(M, N, kp, s, lower, tri, count, max_split) <
           std::tie(o.M, o.N, o.kp, o.s, o.lower, o.tri, o.count, o.max_split);
  }
};
struct TuneVal {
  int bn, splits;
  float ms_best, ms_heuristic;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune;
std::atomic<int> g_autotune{0};

struct TcPlan {
  int bn, splits, per;
};

static cudaError_t tc_run_plan(const TcOperand& A, const TcOperand& B, TcArgs a, const TcPlan& p, int M, int N,
                               double alpha, double beta, double* C, long long ldc, bool lower_only, double* partial,
                               double mma, cudaStream_t st, const TcBatch& bt) {
  a.k_per_split = p.per;
  if (p.splits > 1) {
    a.partial = partial;
    cudaError_t e = p.bn == 16   ? tc_launch<16, 1, EPI_F64>(A, B, a, p.splits, bt.count, mma, st)
                    : p.bn == 64 ? tc_launch<64, 1, EPI_F64>(A, B, a, p.splits, bt.count, mma, st)
                                 : tc_launch<128, 1, EPI_F64>(A, B, a, p.splits, bt.count, mma, st);
    if (e != cudaSuccess) return e;
    return launch_splitk_reduce(partial, p.splits, M, N, alpha, beta, C, ldc, lower_only, TC_BM, st, bt.count,
                                bt.c_stride);
  }
  a.partial = nullptr;
  return p.bn == 16   ? tc_launch<16, 1, EPI_F64>(A, B, a, 1, bt.count, mma, st)
         : p.bn == 64 ? tc_launch<64, 1, EPI_F64>(A, B, a, 1, bt.count, mma, st)
                      : tc_launch<128, 1, EPI_F64>(A, B, a, 1, bt.count, mma, st);
}

static TcPlan plan_for(int k_iters, int splits_wanted, int bn) {
  TcPlan p;
  p.bn = bn;
  p.per = (k_iters + splits_wanted - 1) / splits_wanted;
  p.splits = (k_iters + p.per - 1) / p.per;
  return p;
}

cudaError_t tc_gemm_f64_batched(const TcOperand& A, const TcOperand& B, int M, int N, double alpha, double beta,
                                double* C, long long ldc, bool lower_only, bool tri_b, double* partial, int max_split,
                                int num_sms, unsigned* status, cudaStream_t st, const TcBatch& bt) {
  if (M <= 0 || N <= 0 || bt.count <= 0) return cudaSuccess;
  if (A.s != B.s || A.kp != B.kp || A.kp % TC_BK) return cudaErrorInvalidValue;
  if (lower_only && M != N) return cudaErrorInvalidValue;
  TcArgs a{};
  a.M = M;
  a.N = N;
  a.a_rows_pad = A.rows_pad;
  a.b_rows_pad = B.rows_pad;
  a.s = A.s;
  a.k_iters = A.kp / TC_BK;
  a.lower_only = lower_only ? 1 : 0;
  a.tri_b = tri_b ? 1 : 0;
  a.alpha = alpha;
  a.beta = beta;
  a.C = C;
  a.ldc = ldc;
  a.status = status;
  a.a_brows = bt.a_rows;
  a.b_brows = bt.b_rows;
  a.c_bstride = bt.c_stride;
  const int tm = (M + TC_BM - 1) / TC_BM, tn = (N + 127) / 128;
  const int tiles = (lower_only ? tm * (tm + 1) / 2 : tm * tn) * bt.count;
  const bool can_split = partial && !tri_b;
  int splits = 1, per = a.k_iters;
  if (can_split) split_k(a.k_iters, tiles, num_sms, max_split, splits, per);
  // a narrow B (at most 16 columns, the probe blocks of the apply): 128 x 16
  // tiles, so the MMAs do not run on padding columns
  const int bn0 = (!lower_only && N <= 16) ? 16 : 128;
  TcPlan plan{bn0, splits, per};
  // BF16 MMA flops of the s (s + 1) / 2 slice products over the outputs the
  // method needs (lower triangle of a SYRK; k <= n under tri_b)
  const double prods = 0.5 * a.s * (a.s + 1);
  const double kk = (double)A.kp;
  const double outk = lower_only ? 0.5 * M * (M + 1.0) * kk
                      : tri_b    ? (double)M * 0.5 * N * (N + 1.0)
                                 : (double)M * N * kk;
  const double mma = 2.0 * prods * outk * bt.count;
  const TuneKey key{M, N, A.kp, a.s, a.lower_only, a.tri_b, bt.count, can_split ? max_split : 1};
  bool tuned = false;
  {
    std::lock_guard<std::mutex> g(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      plan = plan_for(a.k_iters, it->second.splits, it->second.bn);
      tuned = true;
    }
  }
  if (!tuned && g_autotune.load() == 2 && !tl_capture) {
    // the narrowest tile wherever it is allowed, heuristic splits, no timing:
    // runs every tile path of a workload (tests)
    plan = plan_for(a.k_iters, splits, lower_only ? 128 : (N <= 16 ? 16 : 64));
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune[key] = TuneVal{plan.bn, plan.splits, 0.0f, 0.0f};
  } else if (!tuned && g_autotune.load() == 1 && !tl_capture && beta == 0.0) {
    // candidates: (tile width, splits), the heuristic first
    const int acc =
        can_split ? std::min(max_split, (a.k_iters + kTcMaxChunksPerSplit - 1) / kTcMaxChunksPerSplit) : 1;
    std::vector<TcPlan> cand;
    auto add = [&](int sp, int bn) {
      if (sp < acc || sp < 1 || sp > a.k_iters || (sp > 1 && !can_split) || (can_split && sp > max_split)) return;
      if (bn == 64 && lower_only) return;
      const TcPlan p = plan_for(a.k_iters, sp, bn);
      for (const TcPlan& q : cand)
        if (q.bn == p.bn && q.splits == p.splits) return;
      cand.push_back(p);
    };
    for (int bn : {bn0, 128, 64}) {
      add(splits, bn);
      add(splits * 2, bn);
      add(splits / 2, bn);
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 1e30f, heur = 0.0f;
    TcPlan best_plan = plan;
    for (size_t i = 0; i < cand.size() && e == cudaSuccess; ++i) {
      e = tc_run_plan(A, B, a, cand[i], M, N, alpha, beta, C, ldc, lower_only, partial, mma, st, bt);  // warm
      if (e == cudaSuccess) e = cudaEventRecord(e0, st);
      for (int r = 0; r < 2 && e == cudaSuccess; ++r)
        e = tc_run_plan(A, B, a, cand[i], M, N, alpha, beta, C, ldc, lower_only, partial, mma, st, bt);
      if (e == cudaSuccess) e = cudaEventRecord(e1, st);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.0f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) break;
      ms *= 0.5f;
      if (i == 0) heur = ms;
      if (ms < best) {
        best = ms;
        best_plan = cand[i];
      }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return e;
    plan = best_plan;
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune[key] = TuneVal{plan.bn, plan.splits, best, heur};
  }
  return tc_run_plan(A, B, a, plan, M, N, alpha, beta, C, ldc, lower_only, partial, mma, st, bt);
}

cudaError_t tc_gemm_f64(const TcOperand& A, const TcOperand& B, int M, int N, double alpha, double beta, double* C,
                        long long ldc, bool lower_only, bool tri_b, double* partial, int max_split, int num_sms,
                        unsigned* status, cudaStream_t st) {
  return tc_gemm_f64_batched(A, B, M, N, alpha, beta, C, ldc, lower_only, tri_b, partial, max_split, num_sms, status,
                             st, TcBatch{1, 0, 0, 0});
}

cudaError_t tc_scaled_slices(const TcOperand& A, const TcOperand& B, int M, int N, const float* colscale,
                             long long cs_bstride, __nv_bfloat16* zs, int zs_rows_pad, int zs_kp, long long zs_bstride,
                             unsigned* status, cudaStream_t st, const TcBatch& bt) {
  if (M <= 0 || N <= 0 || bt.count <= 0) return cudaSuccess;
  if (A.s != B.s || A.kp != B.kp || A.kp % TC_BK || (zs_kp % 8) || (zs_bstride % 8)) return cudaErrorInvalidValue;
  TcArgs a{};
  a.M = M;
  a.N = N;
  a.a_rows_pad = A.rows_pad;
  a.b_rows_pad = B.rows_pad;
  a.s = A.s;
  a.k_iters = A.kp / TC_BK;
  a.k_per_split = a.k_iters;
  a.alpha = 1.0;
  a.status = status;
  a.a_brows = bt.a_rows;
  a.b_brows = bt.b_rows;
  a.zs = zs;
  a.zs_rows_pad = zs_rows_pad;
  a.zs_kp = zs_kp;
  a.zs_bstride = zs_bstride;
  a.colscale = colscale;
  a.cs_bstride = cs_bstride;
  const double mma = 2.0 * 0.5 * a.s * (a.s + 1) * (double)M * N * (double)A.kp * bt.count;
  return tc_launch<128, 1, EPI_SCALE_SLICES>(A, B, a, 1, bt.count, mma, st);
}

cudaError_t tc_gemm_f64_slices(const TcOperand& A, const TcOperand& B, int M, int N, double* C, long long ldc,
                               bool tri_b, __nv_bfloat16* zs, int zs_rows_pad, int zs_kp, __nv_bfloat16* zt,
                               int zt_rows_pad, int zt_kp, unsigned* status, cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (A.s != B.s || A.kp != B.kp || A.kp % TC_BK || (zs_kp % 8) || M > zt_kp || N > zt_rows_pad || M > zs_rows_pad ||
      N > zs_kp)
    return cudaErrorInvalidValue;
  TcArgs a{};
  a.M = M;
  a.N = N;
  a.a_rows_pad = A.rows_pad;
  a.b_rows_pad = B.rows_pad;
  a.s = A.s;
  a.k_iters = A.kp / TC_BK;
  a.k_per_split = a.k_iters;
  a.tri_b = tri_b ? 1 : 0;
  a.alpha = 1.0;
  a.C = C;
  a.ldc = ldc;
  a.zs = zs;
  a.zs_rows_pad = zs_rows_pad;
  a.zs_kp = zs_kp;
  a.zt = zt;
  a.zt_rows_pad = zt_rows_pad;
  a.zt_kp = zt_kp;
  a.status = status;
  const double prods = 0.5 * a.s * (a.s + 1);
  const double outk = tri_b ? (double)M * 0.5 * N * (N + 1.0) : (double)M * N * (double)A.kp;
  return tc_launch<128, 1, EPI_F64_SLICES2>(A, B, a, 1, 1, 2.0 * prods * outk, st);
}

cudaError_t tc_facesplit(const TcOperand& A, const TcOperand& B, int M, int N, int kv_iters, double* C,
                         long long ldc, __nv_bfloat16* zs, int zs_rows_pad, int zs_kp, unsigned* status,
                         cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (A.s != B.s || A.kp != B.kp || A.kp % TC_BK) return cudaErrorInvalidValue;
  TcArgs a{};
  a.M = M;
  a.N = N;
  a.a_rows_pad = A.rows_pad;
  a.b_rows_pad = B.rows_pad;
  a.s = A.s;
  a.k_iters = A.kp / TC_BK;
  a.k_per_split = a.k_iters;
  a.kv_iters = kv_iters;
  a.alpha = 1.0;
  a.C = C;
  a.ldc = ldc;
  a.zs = zs;
  a.zs_rows_pad = zs_rows_pad;
  a.zs_kp = zs_kp;
  a.status = status;
  a.splits = 1;
  const double mma = 2.0 * 0.5 * a.s * (a.s + 1) * (double)M * N * (double)A.kp;
  if (zs) return tc_launch<128, 2, EPI_HAD_SLICES>(A, B, a, 1, 1, mma, st);
  return tc_launch<128, 2, EPI_HAD_F64>(A, B, a, 1, 1, mma, st);
}

}  // namespace isdf

// ---- tile autotuner: C ABI (declared in include/isdf_smw.h)
extern "C" int isdf_set_autotune(int on) { return isdf::g_autotune.exchange(on == 2 ? 2 : (on ? 1 : 0)); }

extern "C" int isdf_autotune_size(void) {
  std::lock_guard<std::mutex> g(isdf::g_tune_mu);
  return (int)isdf::g_tune.size();
}

extern "C" int isdf_autotune_entry(int i, int* key, int* choice, double* ms) {
  std::lock_guard<std::mutex> g(isdf::g_tune_mu);
  if (i < 0 || i >= (int)isdf::g_tune.size()) return -1;
  auto it = isdf::g_tune.begin();
  std::advance(it, i);
  const isdf::TuneKey& k = it->first;
  const int kv[8] = {k.M, k.N, k.kp, k.s, k.lower, k.tri, k.count, k.max_split};
  if (key)
    for (int j = 0; j < 8; ++j) key[j] = kv[j];
  if (choice) {
    choice[0] = it->second.bn;
    choice[1] = it->second.splits;
  }
  if (ms) {
    ms[0] = it->second.ms_best;
    ms[1] = it->second.ms_heuristic;
  }
  return 0;
}

extern "C" void isdf_autotune_clear(void) {
  std::lock_guard<std::mutex> g(isdf::g_tune_mu);
  isdf::g_tune.clear();
}

