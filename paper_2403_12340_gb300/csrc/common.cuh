// Shared device helpers for the ISDF-SMW kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace isdf {

// Device status bits, OR-ed into a status word by kernels.
enum : unsigned {
  ST_NONFINITE = 1u,   // a NaN / Inf was seen in an input
  ST_NOT_SPD = 2u,     // non-positive pivot in an unpivoted Cholesky
  ST_TIMEOUT = 4u,     // a bounded device-side wait gave up
  ST_BADINDEX = 8u,    // an index failed a device-side bounds check
};

// 1 / d: an FP32 estimate from the leading bits of d (integer operations and
// one FP32 reciprocal), then two Newton steps y <- y + y (1 - d y) in FP64
// (4 FP64 instructions on the chain, no conversion on the FP64 pipe).
__device__ __forceinline__ double recip_newton(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const int ef = (int)((b >> 52) & 0x7FFull) - 1023 + 127;
  if (ef <= 1 || ef >= 253) return 1.0 / d;  // outside the FP32 range of the estimate
  const float df = __uint_as_float((unsigned)((b >> 63) << 31) | ((unsigned)ef << 23) | (unsigned)((b >> 29) & 0x7FFFFFull));
  const unsigned yb = __float_as_uint(__frcp_rn(df));  // a normal float: 2 <= its biased exponent <= 252
  double y = __longlong_as_double((long long)(((unsigned long long)(yb >> 31) << 63) |
                                              ((unsigned long long)(((yb >> 23) & 0xFFu) - 127 + 1023) << 52) |
                                              ((unsigned long long)(yb & 0x7FFFFFu) << 29)));
  double e = fma(-d, y, 1.0);
  y = fma(y, e, y);
  e = fma(-d, y, 1.0);
  return fma(y, e, y);
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier for cooperative launches (all blocks co-resident).
// A block records the generation before arriving; the last arriver resets
// the counter and bumps the generation.  The wait is bounded by `limit_ns`
// of wall time: on expiry the status word gets ST_TIMEOUT and the barrier
// returns false, so the caller leaves the kernel instead of hanging.
struct GridBarrier {
  unsigned* count;
  unsigned* gen;
};

__device__ __forceinline__ bool grid_sync(GridBarrier b, unsigned* status, uint64_t limit_ns) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    unsigned my_gen = ld_acquire(b.gen);
    __threadfence();
    unsigned arrived = atomicAdd(b.count, 1u);
    if (arrived == gridDim.x * gridDim.y * gridDim.z - 1u) {
      atomicExch(b.count, 0u);
      __threadfence();
      atomicAdd(b.gen, 1u);
    } else {
      uint64_t t0 = global_ns();
      unsigned spins = 0;
      while (ld_acquire(b.gen) == my_gen) {
        if ((++spins & 255u) == 0u) {
          if (global_ns() - t0 > limit_ns || (ld_acquire(status) & ST_TIMEOUT)) {
            atomicOr(status, ST_TIMEOUT);
            ok = 0;
            break;
          }
        }
        __nanosleep(20);
      }
    }
    __threadfence();
    s_ok = ok && !(ld_acquire(status) & ST_TIMEOUT);
  }
  __syncthreads();
  return s_ok != 0;
}

// ---------------------------------------------------------------------------
// FP64 tiled GEMM engine: acc(m, n) += sum_k A(m, k) B(n, k) on a BM x BN
// output tile, 16-deep k slices staged in padded shared memory, a TM x TN
// register tile per thread.  Thread t owns rows m0 + tx + (BM/TM) i and
// columns n0 + ty + (BN/TN) j with tx = t % (BM/TM), ty = t / (BM/TM), so
// column-major stores of a tile are coalesced along m.  FP64 on GB300 is
// bound by the DFMA pipe (measured 1.2 TFLOP/s per GPU); one shared-memory
// load feeds TN (resp. TM) DFMAs, which keeps that pipe saturated.
// ---------------------------------------------------------------------------
constexpr int GT_BK = 16;

// Operand accessor: element (row, k) of a matrix operand with `rows` rows.
// KCONTIG = false: row index contiguous, address p[row + ld * k].
// KCONTIG = true : k index contiguous,   address p[k + ld * row].
template <bool KCONTIG>
struct Operand {
  static constexpr bool kcontig = KCONTIG;
  const double* p;
  long long ld;
  int rows;
  __device__ __forceinline__ double get(int row, int k) const {
    return KCONTIG ? p[(long long)row * ld + k] : p[row + ld * (long long)k];
  }
};

// ---- double-float helpers (the mixed path's FP64-grade work on the FP32 pipe) ----

// An FP32 value as FP64 from its bit fields (exact for normal values; zero
// and subnormals give a signed zero, infinities and NaN stay what they are).
__device__ __forceinline__ double f32_as_f64(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned ex = (b >> 23) & 0xffu;
  const unsigned long long sgn = (unsigned long long)(b & 0x80000000u) << 32;
  if (ex == 0) return __longlong_as_double((long long)sgn);
  const unsigned long long e64 = ex == 0xffu ? 0x7ffull : (unsigned long long)(ex + 896u);  // 1023 - 127
  return __longlong_as_double((long long)(sgn | (e64 << 52) | ((unsigned long long)(b & 0x7fffffu) << 29)));
}

// x = hi + lo to 48 significant bits
__device__ __forceinline__ float2 split_f64(double x) {
  const float h = __double2float_rn(x);
  return make_float2(h, __double2float_rn(x - f32_as_f64(h)));
}

// FP64 -> FP32 rounded to nearest even by integer operations on the bit
// fields (no FP64-pipe conversion; GB300 issues FP64 instructions, which
// include the conversions, at 1/64 of the FP32 rate).  Results below the
// FP32 normal range flush to zero, above it become infinity.
__device__ __forceinline__ float f64_to_f32_rn(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int sign = (unsigned int)(b >> 63) << 31;
  const int ef = (int)((b >> 52) & 0x7FFull) - 1023 + 127;
  if (ef <= 0) return __uint_as_float(sign);
  if (ef >= 255) return __uint_as_float(sign | 0x7F800000u);
  const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  const unsigned int rem = (unsigned int)(m & 0x1FFFFFFFull);
  unsigned int bits = ((unsigned int)ef << 23) | (unsigned int)(m >> 29);
  if (rem > 0x10000000u || (rem == 0x10000000u && (bits & 1u))) bits += 1u;  // a carry moves into the exponent
  return __uint_as_float(sign | bits);
}

// split_f64 with one FP64 instruction (the subtraction) instead of three
__device__ __forceinline__ float2 split_f64_fast(double x) {
  const float h = f64_to_f32_rn(x);
  return make_float2(h, f64_to_f32_rn(x - f32_as_f64(h)));
}

// (hi, lo) += a b: the product's exact FP32 error and both cross terms go to
// lo (a.lo b.lo, 2^-48 relative, is dropped); hi + p by Knuth's two-sum.
// The _rn intrinsics keep the compiler from fusing the error-free steps.
__device__ __forceinline__ void df_fma(float2 a, float2 b, float& hi, float& lo) {
  const float p = __fmul_rn(a.x, b.x);
  float e = fmaf(a.x, b.x, -p);
  e = fmaf(a.x, b.y, e);
  e = fmaf(a.y, b.x, e);
  const float s = __fadd_rn(hi, p);
  const float v = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, v)), __fsub_rn(p, v));
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(err, e));
}

// (hi, lo) <- hi + lo renormalised (|hi| >= |lo| or hi = 0 after a chunk)
__device__ __forceinline__ void df_renorm(float& hi, float& lo) {
  const float s = __fadd_rn(hi, lo);
  lo = __fsub_rn(lo, __fsub_rn(s, hi));
  hi = s;
}

// ---- double-float scalar arithmetic (latency-bound chains on the FP32 pipe) ----
// A value is a float2 (x = hi, y = lo) with |lo| <= ulp(hi) / 2 after df_norm.

__device__ __forceinline__ float2 df_norm(float hi, float lo) {
  const float s = __fadd_rn(hi, lo);
  return make_float2(s, __fsub_rn(lo, __fsub_rn(s, hi)));
}

__device__ __forceinline__ double df_to_f64(float2 a) { return f32_as_f64(a.x) + f32_as_f64(a.y); }

// a b to about 2^-47 relative (a.lo b.lo dropped)
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = fmaf(a.x, b.x, -p);
  e = fmaf(a.x, b.y, e);
  e = fmaf(a.y, b.x, e);
  return df_norm(p, e);
}

// c - a b, with the sum by Knuth's two-sum
__device__ __forceinline__ float2 df_fms(float2 c, float2 a, float2 b) {
  float hi = c.x, lo = c.y;
  df_fma(make_float2(-a.x, -a.y), b, hi, lo);
  return df_norm(hi, lo);
}

// 1 / sqrt(d): the FP32 estimate, then one Newton step y + y (1 - d y^2) / 2
// with d y^2 in double-float (about 2^-46 relative)
__device__ __forceinline__ float2 df_rsqrt(float2 d) {
  const float y = rsqrtf(d.x);
  const float2 y2 = make_float2(__fmul_rn(y, y), fmaf(y, y, -__fmul_rn(y, y)));
  const float2 t = df_mul(d, y2);  // about 1
  const float e = __fsub_rn(__fsub_rn(1.0f, t.x), t.y);
  return df_norm(y, __fmul_rn(__fmul_rn(0.5f, y), e));
}

// 1 / d: the correctly rounded FP32 reciprocal of d.hi, then one Newton step
// r + r (1 - d r) with the residual 1 - d r formed exactly from an FMA (the
// step doubles the 24 correct bits to about 47).
__device__ __forceinline__ float2 df_recip(float2 d) {
  const float r = __frcp_rn(d.x);
  const float p = __fmul_rn(d.x, r);
  const float pe = fmaf(d.x, r, -p);
  const float e = fmaf(-d.y, r, __fsub_rn(__fsub_rn(1.0f, p), pe));
  return df_norm(r, __fmul_rn(r, e));
}

template <int BM, int BN, int TM, int TN>
struct Tile {
  static constexpr int kBM = BM, kBN = BN, kTM = TM, kTN = TN;
  static constexpr int XT = BM / TM, YT = BN / TN, NT = XT * YT;
  struct Smem {
    double a[GT_BK][BM + 1];
    double b[GT_BK][BN + 1];
  };
  struct SmemDf {  // the same tiles as float pairs (double-float mode)
    float2 a[GT_BK][BM + 1];
    float2 b[GT_BK][BN + 1];
  };
};

using TileSq = Tile<64, 64, 4, 4>;       // 256 threads, square tiles
using TileSm = Tile<32, 32, 2, 2>;       // 256 threads, small square tiles (short GEMMs)
using TileNarrow = Tile<128, 16, 4, 2>;  // 256 threads, tall-skinny (probe blocks)

// sm[k][row] = op(row0 + row, k0 + k), zero outside [0, rows) x [k0, kend).
template <int NT, int ROWS, class Op>
__device__ __forceinline__ void load_slice(double (*sm)[ROWS + 1], const Op& op, int row0, int k0,
                                           int kend) {
  const int t = threadIdx.x;
  constexpr int PER = (ROWS * GT_BK + NT - 1) / NT;
#pragma unroll
  for (int s = 0; s < PER; ++s) {
    int idx = t + s * NT;
    if (idx >= ROWS * GT_BK) break;
    int r, k;
    if (!Op::kcontig) {
      r = idx % ROWS;
      k = idx / ROWS;
    } else {
      k = idx % GT_BK;
      r = idx / GT_BK;
    }
    int gr = row0 + r, gk = k0 + k;
    sm[k][r] = (gr < op.rows && gk < kend) ? op.get(gr, gk) : 0.0;
  }
}

template <class T>
__device__ __forceinline__ void mma_slice(double (&acc)[T::kTM][T::kTN], const typename T::Smem& s) {
  const int tx = threadIdx.x % T::XT, ty = threadIdx.x / T::XT;
#pragma unroll
  for (int kk = 0; kk < GT_BK; ++kk) {
    double a[T::kTM], b[T::kTN];
#pragma unroll
    for (int i = 0; i < T::kTM; ++i) a[i] = s.a[kk][tx + T::XT * i];
#pragma unroll
    for (int j = 0; j < T::kTN; ++j) b[j] = s.b[kk][ty + T::YT * j];
#pragma unroll
    for (int i = 0; i < T::kTM; ++i)
#pragma unroll
      for (int j = 0; j < T::kTN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
  }
}

// acc += sum_{k in [kbeg, kend)} A(m0 + ., k) B(n0 + ., k)
template <class T, class OpA, class OpB>
__device__ __forceinline__ void gemm_mainloop(double (&acc)[T::kTM][T::kTN], typename T::Smem& s,
                                              const OpA& A, const OpB& B, int m0, int n0, int kbeg,
                                              int kend) {
  for (int k0 = kbeg; k0 < kend; k0 += GT_BK) {
    load_slice<T::NT, T::kBM>(s.a, A, m0, k0, kend);
    load_slice<T::NT, T::kBN>(s.b, B, n0, k0, kend);
    __syncthreads();
    mma_slice<T>(acc, s);
    __syncthreads();
  }
}

// The double-float form of the main loop: each operand element is split
// into a float pair as it is staged (hi = fl32(x), lo = fl32(x - hi)), the
// products accumulate in (hi, lo) pairs on the FP32 pipe (df_fma),
// renormalised after every K slice, and acc = hi + lo in FP64 at the end
// (about 2^-46 relative per product sum instead of 2^-53).
template <int NT, int ROWS, class Op>
__device__ __forceinline__ void load_slice_df(float2 (*sm)[ROWS + 1], const Op& op, int row0, int k0, int kend) {
  const int t = threadIdx.x;
  constexpr int PER = (ROWS * GT_BK + NT - 1) / NT;
#pragma unroll
  for (int s = 0; s < PER; ++s) {
    int idx = t + s * NT;
    if (idx >= ROWS * GT_BK) break;
    int r, k;
    if (!Op::kcontig) {
      r = idx % ROWS;
      k = idx / ROWS;
    } else {
      k = idx % GT_BK;
      r = idx / GT_BK;
    }
    int gr = row0 + r, gk = k0 + k;
    sm[k][r] = (gr < op.rows && gk < kend) ? split_f64(op.get(gr, gk)) : make_float2(0.0f, 0.0f);
  }
}

template <class T, class OpA, class OpB>
__device__ __forceinline__ void gemm_mainloop_df(double (&acc)[T::kTM][T::kTN], typename T::SmemDf& s,
                                                 const OpA& A, const OpB& B, int m0, int n0, int kbeg,
                                                 int kend) {
  const int tx = threadIdx.x % T::XT, ty = threadIdx.x / T::XT;
  float hi[T::kTM][T::kTN], lo[T::kTM][T::kTN];
#pragma unroll
  for (int i = 0; i < T::kTM; ++i)
#pragma unroll
    for (int j = 0; j < T::kTN; ++j) hi[i][j] = lo[i][j] = 0.0f;
  for (int k0 = kbeg; k0 < kend; k0 += GT_BK) {
    load_slice_df<T::NT, T::kBM>(s.a, A, m0, k0, kend);
    load_slice_df<T::NT, T::kBN>(s.b, B, n0, k0, kend);
    __syncthreads();
#pragma unroll 2
    for (int kk = 0; kk < GT_BK; ++kk) {
      float2 a[T::kTM], b[T::kTN];
#pragma unroll
      for (int i = 0; i < T::kTM; ++i) a[i] = s.a[kk][tx + T::XT * i];
#pragma unroll
      for (int j = 0; j < T::kTN; ++j) b[j] = s.b[kk][ty + T::YT * j];
#pragma unroll
      for (int i = 0; i < T::kTM; ++i)
#pragma unroll
        for (int j = 0; j < T::kTN; ++j) df_fma(a[i], b[j], hi[i][j], lo[i][j]);
    }
#pragma unroll
    for (int i = 0; i < T::kTM; ++i)
#pragma unroll
      for (int j = 0; j < T::kTN; ++j) df_renorm(hi[i][j], lo[i][j]);
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < T::kTM; ++i)
#pragma unroll
    for (int j = 0; j < T::kTN; ++j) acc[i][j] = f32_as_f64(hi[i][j]) + f32_as_f64(lo[i][j]);
}

template <class T>
__device__ __forceinline__ void zero_acc(double (&acc)[T::kTM][T::kTN]) {
#pragma unroll
  for (int i = 0; i < T::kTM; ++i)
#pragma unroll
    for (int j = 0; j < T::kTN; ++j) acc[i][j] = 0.0;
}

// (row, col) of register element (i, j) of this thread in tile (m0, n0).
template <class T>
__device__ __forceinline__ int tile_row(int m0, int i) {
  return m0 + (int)(threadIdx.x % T::XT) + T::XT * i;
}
template <class T>
__device__ __forceinline__ int tile_col(int n0, int j) {
  return n0 + (int)(threadIdx.x / T::XT) + T::YT * j;
}

// Map a linear block index onto lower-triangular tile coordinates (mt >= nt).
__device__ __forceinline__ void lower_tile(int lin, int& mt, int& nt) {
  int m = (int)((sqrt(8.0 * (double)lin + 1.0) - 1.0) * 0.5);
  while ((m + 1) * (m + 2) / 2 <= lin) ++m;
  while (m * (m + 1) / 2 > lin) --m;
  mt = m;
  nt = lin - m * (m + 1) / 2;
}

}  // namespace isdf
