// Batched 3-D real FFTs on the periodic grid, written for the Coulomb
// operator of the ISDF-SMW path (V = F^-1 diag(v_G / dV) F; Algorithm 3
// step 2 applies it to the interpolation vectors).  No cuFFT.
//
// Two kernels per direction:
//   xy kernel: one thread block per (column, z plane).  The real n1 x n2
//     plane is loaded into shared memory with lines y = 2t and 2t+1 packed
//     as one complex line, transformed along x, unpacked to the half
//     spectrum kx = 0..n1/2 (Hermitian symmetry of a real line), then
//     transformed along y.  The inverse runs the same steps backwards.
//   z kernel: one thread block per (column, 32 consecutive (ky, kx)
//     positions); transforms along z and multiplies by a real weight table
//     (for the convolution: forward, weight, inverse in one pass).
// 1-D transforms are Stockham auto-sort passes with radices 4, 2, 3, 5 (and
// a direct DFT for 7, 11, 13), ping-ponging between two shared buffers.
// Twiddles exp(-2 pi i t / n) come from a per-axis table computed on the
// host in float64.
#include <cuda_bf16.h>

#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace isdf {

constexpr int FFT_THREADS = 256;
constexpr int FFT_ZCHUNK = 32;

// Complex arithmetic for both precisions (double2 for the FP64 path, float2
// for the mixed path); twiddle tables are float64 and are rounded on load.
template <class C>
struct Real;
template <>
struct Real<double2> {
  using T = double;
};
template <>
struct Real<float2> {
  using T = float;
};
template <class C>
__device__ __forceinline__ C mk(typename Real<C>::T x, typename Real<C>::T y) {
  C c;
  c.x = x;
  c.y = y;
  return c;
}
template <class C>
__device__ __forceinline__ C cmul(C a, C b) {
  return mk<C>(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
template <class C>
__device__ __forceinline__ C cadd(C a, C b) {
  return mk<C>(a.x + b.x, a.y + b.y);
}
template <class C>
__device__ __forceinline__ C csub(C a, C b) {
  return mk<C>(a.x - b.x, a.y - b.y);
}
// FP64 input to the transform precision; for FP32 by integer operations
// (no FP64 instruction: GB300's FP64 pipe is 1/64 rate).
template <class T>
__device__ __forceinline__ T to_real(double x);
template <>
__device__ __forceinline__ double to_real<double>(double x) {
  return x;
}
template <>
__device__ __forceinline__ float to_real<float>(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int sign = (unsigned int)(b >> 63) << 31;
  const int ef = (int)((b >> 52) & 0x7FFull) - 1023 + 127;
  if (ef <= 0) return __uint_as_float(sign);
  if (ef >= 255) return __uint_as_float(sign | 0x7F800000u);
  const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  const unsigned int rem = (unsigned int)(m & 0x1FFFFFFFull);
  unsigned int bits = ((unsigned int)ef << 23) | (unsigned int)(m >> 29);
  if (rem > 0x10000000u || (rem == 0x10000000u && (bits & 1u))) bits += 1u;
  return __uint_as_float(sign | bits);
}

template <class C>
__device__ __forceinline__ C from_tw(const double2 w) {
  return mk<C>((typename Real<C>::T)w.x, (typename Real<C>::T)w.y);
}

// twiddle exp(DIR 2 pi i t / n) with DIR = -1 forward, +1 inverse
template <int DIR, class C>
__device__ __forceinline__ C twid(const C* tw, int t) {
  C w = tw[t];
  if (DIR > 0) w.y = -w.y;
  return w;
}

template <int DIR, class C>
__device__ __forceinline__ void bfly2(C* v) {
  C a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}

template <int DIR, class C>
__device__ __forceinline__ void bfly3(C* v) {
  using T = typename Real<C>::T;
  const T s3 = (T)0.86602540378443864676;  // sqrt(3) / 2
  const T h = (T)0.5;
  C t1 = cadd(v[1], v[2]);
  C t2 = mk<C>(v[0].x - h * t1.x, v[0].y - h * t1.y);
  C m = mk<C>(s3 * (v[1].x - v[2].x), s3 * (v[1].y - v[2].y));
  v[0] = cadd(v[0], t1);
  if (DIR < 0) {  // X1 = t2 - i m, X2 = t2 + i m
    v[1] = mk<C>(t2.x + m.y, t2.y - m.x);
    v[2] = mk<C>(t2.x - m.y, t2.y + m.x);
  } else {
    v[1] = mk<C>(t2.x - m.y, t2.y + m.x);
    v[2] = mk<C>(t2.x + m.y, t2.y - m.x);
  }
}

template <int DIR, class C>
__device__ __forceinline__ void bfly4(C* v) {
  C a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
  C c = cadd(v[1], v[3]), d = csub(v[1], v[3]);
  v[0] = cadd(a, c);
  v[2] = csub(a, c);
  if (DIR < 0) {  // X1 = b - i d, X3 = b + i d
    v[1] = mk<C>(b.x + d.y, b.y - d.x);
    v[3] = mk<C>(b.x - d.y, b.y + d.x);
  } else {
    v[1] = mk<C>(b.x - d.y, b.y + d.x);
    v[3] = mk<C>(b.x + d.y, b.y - d.x);
  }
}

// direct R-point DFT with table twiddles (w_R^m = tw[(m mod R) n / R])
template <int R, int DIR, class C>
__device__ __forceinline__ void bfly_direct(C* v, const C* tw, int n) {
  C out[R];
  const int step = n / R;
#pragma unroll
  for (int a = 0; a < R; ++a) {
    C acc = v[0];
#pragma unroll
    for (int b = 1; b < R; ++b) acc = cadd(acc, cmul(v[b], twid<DIR>(tw, ((a * b) % R) * step)));
    out[a] = acc;
  }
#pragma unroll
  for (int a = 0; a < R; ++a) v[a] = out[a];
}

template <int R, int DIR, class C>
__device__ __forceinline__ void bfly(C* v, const C* tw, int n) {
  if constexpr (R == 2) bfly2<DIR>(v);
  else if constexpr (R == 3) bfly3<DIR>(v);
  else if constexpr (R == 4) bfly4<DIR>(v);
  else bfly_direct<R, DIR>(v, tw, n);
}

// One Stockham pass of radix R over `nlines` lines of length n (element e of
// line l at buf[l * sl + e * se]); Ns = product of the radices done so far.
template <int R, int DIR, class C>
__device__ __forceinline__ void stockham_pass(const C* __restrict__ src, C* __restrict__ dst, int n, int Ns,
                                              int nlines, int se, int sl, const C* tw) {
  const int nR = n / R;
  const int tstep = n / (Ns * R);
  for (int idx = threadIdx.x; idx < nlines * nR; idx += blockDim.x) {
    // consecutive threads on consecutive addresses: along the line where its
    // elements are adjacent (se == 1), across the lines where the lines are
    // (sl == 1, the y pass of a plane), which keeps shared-memory banks apart
    int line, j;
    if (sl == 1 && se != 1) {
      j = idx / nlines;
      line = idx - j * nlines;
    } else {
      line = idx / nR;
      j = idx - line * nR;
    }
    int k = j % Ns;
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src[line * sl + (j + r * nR) * se];
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = cmul(v[r], twid<DIR>(tw, r * k * tstep));
    }
    bfly<R, DIR>(v, tw, n);
    int base = (j / Ns) * Ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[line * sl + (base + r * Ns) * se] = v[r];
  }
}

// 1-D transforms of all lines; returns the buffer holding the result.
template <int DIR, class C>
__device__ C* fft_lines(C* src, C* dst, const FftAxis& ax, const C* tw, int nlines, int se, int sl) {
  int Ns = 1;
  const int n = ax.n;
  for (int f = 0; f < ax.nf; ++f) {
    int R = ax.f[f];
    switch (R) {
      case 2: stockham_pass<2, DIR>(src, dst, n, Ns, nlines, se, sl, tw); break;
      case 3: stockham_pass<3, DIR>(src, dst, n, Ns, nlines, se, sl, tw); break;
      case 4: stockham_pass<4, DIR>(src, dst, n, Ns, nlines, se, sl, tw); break;
      case 5: stockham_pass<5, DIR>(src, dst, n, Ns, nlines, se, sl, tw); break;
      case 7: stockham_pass<7, DIR>(src, dst, n, Ns, nlines, se, sl, tw); break;
      case 11: stockham_pass<11, DIR>(src, dst, n, Ns, nlines, se, sl, tw); break;
      default: stockham_pass<13, DIR>(src, dst, n, Ns, nlines, se, sl, tw); break;
    }
    __syncthreads();
    C* t = src;
    src = dst;
    dst = t;
    Ns *= R;
  }
  return src;
}

// ---- compile-time transform length ---------------------------------------
// With the length known at compile time every index division in the passes
// becomes a multiplication by a constant and the pass loop unrolls.
__host__ __device__ constexpr int first_radix(int n) {
  return n % 4 == 0 ? 4 : n % 2 == 0 ? 2 : n % 3 == 0 ? 3 : n % 5 == 0 ? 5 : n % 7 == 0 ? 7 : n % 11 == 0 ? 11 : 13;
}

template <int N, int NS, int REM, int DIR, class C>
__device__ __forceinline__ C* fft_lines_ct(C* src, C* dst, const C* tw, int nlines, int se, int sl) {
  if constexpr (REM == 1) {
    return src;
  } else {
    constexpr int R = first_radix(REM);
    stockham_pass<R, DIR>(src, dst, N, NS, nlines, se, sl, tw);
    __syncthreads();
    return fft_lines_ct<N, NS * R, REM / R, DIR>(dst, src, tw, nlines, se, sl);
  }
}

struct XYShape {
  int n1, n2, h, npair, buf;  // buf = complex elements per ping-pong buffer
};

__device__ __forceinline__ XYShape xy_shape(const FftGrid& g) {
  XYShape s;
  s.n1 = g.ax[0].n;
  s.n2 = g.ax[1].n;
  s.h = g.h;
  s.npair = (s.n2 + 1) / 2;
  s.buf = max(s.npair * s.n1, s.h * s.n2);
  return s;
}

// Forward xy: real plane -> half spectrum plane P[ky][kx] (h x n2).  The
// input is float64; the transform runs in the precision of C; the output
// plane is written as C (interleaved re, im) at S + lds * col (in units of
// Real<C>::T).
template <class C>
__global__ void __launch_bounds__(FFT_THREADS) k_fft_xy_fwd(FftGrid g, const double* __restrict__ X, long long ldx,
                                                            typename Real<C>::T* __restrict__ S, long long lds) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  C* sm = reinterpret_cast<C*>(sm_raw);
  using T = typename Real<C>::T;
  const XYShape sh = xy_shape(g);
  C* twx = sm;
  C* twy = twx + sh.n1;
  C* b0 = twy + sh.n2;
  C* b1 = b0 + sh.buf;
  const int z = blockIdx.x, col = blockIdx.y;
  for (int t = threadIdx.x; t < sh.n1; t += blockDim.x) twx[t] = from_tw<C>(((const double2*)g.ax[0].tw)[t]);
  for (int t = threadIdx.x; t < sh.n2; t += blockDim.x) twy[t] = from_tw<C>(((const double2*)g.ax[1].tw)[t]);
  const double* plane = X + ldx * (long long)col + (long long)z * sh.n1 * sh.n2;
  for (int idx = threadIdx.x; idx < sh.npair * sh.n1; idx += blockDim.x) {
    int t = idx / sh.n1, x = idx - t * sh.n1;
    int y0 = 2 * t, y1 = 2 * t + 1;
    double re = plane[x + sh.n1 * y0];
    double im = y1 < sh.n2 ? plane[x + sh.n1 * y1] : 0.0;
    b0[t * sh.n1 + x] = mk<C>(to_real<T>(re), to_real<T>(im));
  }
  __syncthreads();
  C* res = fft_lines<-1>(b0, b1, g.ax[0], twx, sh.npair, 1, sh.n1);
  C* P = (res == b0) ? b1 : b0;
  // unpack: A_k = (Z_k + conj Z_{-k}) / 2, B_k = (Z_k - conj Z_{-k}) / (2 i)
  const T half = (T)0.5;
  for (int idx = threadIdx.x; idx < sh.npair * sh.h; idx += blockDim.x) {
    int t = idx / sh.h, k = idx - t * sh.h;
    C zk = res[t * sh.n1 + k];
    C zm = res[t * sh.n1 + (k == 0 ? 0 : sh.n1 - k)];
    C A = mk<C>(half * (zk.x + zm.x), half * (zk.y - zm.y));
    C B = mk<C>(half * (zk.y + zm.y), -half * (zk.x - zm.x));
    P[(2 * t) * sh.h + k] = A;
    if (2 * t + 1 < sh.n2) P[(2 * t + 1) * sh.h + k] = B;
  }
  __syncthreads();
  C* other = (P == b0) ? b1 : b0;
  C* Q = fft_lines<-1>(P, other, g.ax[1], twy, sh.h, sh.h, 1);
  C* out = (C*)(S + lds * (long long)col) + (long long)z * sh.n2 * sh.h;
  for (int idx = threadIdx.x; idx < sh.n2 * sh.h; idx += blockDim.x) out[idx] = Q[idx];
}

// Inverse xy: half spectrum plane -> real plane, Y = X + result (X may be null).
__global__ void __launch_bounds__(FFT_THREADS) k_fft_xy_inv(FftGrid g, const double* __restrict__ S,
                                                            long long lds, const double* X, long long ldx,
                                                            double* Y, long long ldy) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  double2* sm = reinterpret_cast<double2*>(sm_raw);
  const XYShape sh = xy_shape(g);
  double2* twx = sm;
  double2* twy = twx + sh.n1;
  double2* b0 = twy + sh.n2;
  double2* b1 = b0 + sh.buf;
  const int z = blockIdx.x, col = blockIdx.y;
  for (int t = threadIdx.x; t < sh.n1; t += blockDim.x) twx[t] = ((const double2*)g.ax[0].tw)[t];
  for (int t = threadIdx.x; t < sh.n2; t += blockDim.x) twy[t] = ((const double2*)g.ax[1].tw)[t];
  const double2* in = (const double2*)(S + lds * (long long)col) + (long long)z * sh.n2 * sh.h;
  for (int idx = threadIdx.x; idx < sh.n2 * sh.h; idx += blockDim.x) b0[idx] = in[idx];
  __syncthreads();
  double2* P = fft_lines<1>(b0, b1, g.ax[1], twy, sh.h, sh.h, 1);
  double2* Zb = (P == b0) ? b1 : b0;
  // repack pairs of lines: Z_k = A_k + i B_k over the full k range
  for (int idx = threadIdx.x; idx < sh.npair * sh.n1; idx += blockDim.x) {
    int t = idx / sh.n1, k = idx - t * sh.n1;
    bool lo = k < sh.h;
    int kk = lo ? k : sh.n1 - k;
    double2 A = P[(2 * t) * sh.h + kk];
    double2 B = (2 * t + 1 < sh.n2) ? P[(2 * t + 1) * sh.h + kk] : mk<double2>(0.0, 0.0);
    if (!lo) {
      A.y = -A.y;
      B.y = -B.y;
    }
    Zb[t * sh.n1 + k] = mk<double2>(A.x - B.y, A.y + B.x);
  }
  __syncthreads();
  double2* other = (Zb == b0) ? b1 : b0;
  double2* R = fft_lines<1>(Zb, other, g.ax[0], twx, sh.npair, 1, sh.n1);
  const long long off = (long long)z * sh.n1 * sh.n2;
  for (int idx = threadIdx.x; idx < sh.npair * sh.n1; idx += blockDim.x) {
    int t = idx / sh.n1, x = idx - t * sh.n1;
    double2 v = R[t * sh.n1 + x];
    long long r0 = off + x + (long long)sh.n1 * (2 * t);
    double a0 = X ? X[ldx * (long long)col + r0] : 0.0;
    Y[ldy * (long long)col + r0] = a0 + v.x;
    if (2 * t + 1 < sh.n2) {
      long long r1 = r0 + sh.n1;
      double a1 = X ? X[ldx * (long long)col + r1] : 0.0;
      Y[ldy * (long long)col + r1] = a1 + v.y;
    }
  }
}

// z transforms of FFT_ZCHUNK consecutive (ky, kx) positions of one column.
// MODE 0: forward then multiply by wt, in place.
// MODE 1: forward, multiply, inverse, in place (the Coulomb convolution).
// MODE 2: forward, multiply, then write BF16 slices of the weighted spectrum
//         (slice l at out[(l rows_pad + col) kp + 2 q + {0: re, 1: im}], q the
//         complex index) instead of writing back: the K-major operand of the
//         tensor-core SYRK G = S^T S.
template <int MODE, class C>
__global__ void __launch_bounds__(FFT_THREADS) k_fft_z(FftGrid g, typename Real<C>::T* S, long long lds,
                                                       const double* __restrict__ wt, __nv_bfloat16* out,
                                                       int rows_pad, int kp, int nsl) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  C* sm = reinterpret_cast<C*>(sm_raw);
  using T = typename Real<C>::T;
  const int n3 = g.ax[2].n;
  const int plane = g.ax[1].n * g.h;
  C* twz = sm;
  C* b0 = twz + n3;
  C* b1 = b0 + n3 * FFT_ZCHUNK;
  const int q0 = blockIdx.x * FFT_ZCHUNK, col = blockIdx.y;
  const int nq = min(FFT_ZCHUNK, plane - q0);
  for (int t = threadIdx.x; t < n3; t += blockDim.x) twz[t] = from_tw<C>(((const double2*)g.ax[2].tw)[t]);
  C* base = (C*)(S + lds * (long long)col);  // (twiddles: n3 conversions per block, negligible)
  for (int idx = threadIdx.x; idx < n3 * FFT_ZCHUNK; idx += blockDim.x) {
    int z = idx / FFT_ZCHUNK, c = idx - z * FFT_ZCHUNK;
    b0[idx] = c < nq ? base[(long long)z * plane + q0 + c] : mk<C>((T)0, (T)0);
  }
  __syncthreads();
  C* R = fft_lines<-1>(b0, b1, g.ax[2], twz, FFT_ZCHUNK, FFT_ZCHUNK, 1);
  if (wt) {
    for (int idx = threadIdx.x; idx < n3 * FFT_ZCHUNK; idx += blockDim.x) {
      int z = idx / FFT_ZCHUNK, c = idx - z * FFT_ZCHUNK;
      T w = c < nq ? to_real<T>(wt[(long long)z * plane + q0 + c]) : (T)0;
      R[idx] = mk<C>(R[idx].x * w, R[idx].y * w);
    }
    __syncthreads();
  }
  if (MODE == 1) {
    C* other = (R == b0) ? b1 : b0;
    R = fft_lines<1>(R, other, g.ax[2], twz, FFT_ZCHUNK, FFT_ZCHUNK, 1);
  }
  if (MODE == 2) {
    const long long sstr = (long long)rows_pad * kp;
    for (int idx = threadIdx.x; idx < n3 * FFT_ZCHUNK; idx += blockDim.x) {
      int z = idx / FFT_ZCHUNK, c = idx - z * FFT_ZCHUNK;
      if (c >= nq) continue;
      long long k = 2ll * ((long long)z * plane + q0 + c);
      T v[2] = {R[idx].x, R[idx].y};
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float vf = (float)v[h];  // T is float on this path
        __nv_bfloat16 x0 = __float2bfloat16_rn(vf);
        float r1 = vf - __bfloat162float(x0);
        __nv_bfloat16 x1 = __float2bfloat16_rn(r1);
        __nv_bfloat16 x2 = __float2bfloat16_rn(r1 - __bfloat162float(x1));
        long long o = (long long)col * kp + k + h;
        out[o] = x0;
        if (nsl > 1) out[o + sstr] = x1;
        if (nsl > 2) out[o + 2 * sstr] = x2;
      }
    }
    return;
  }
  for (int idx = threadIdx.x; idx < n3 * FFT_ZCHUNK; idx += blockDim.x) {
    int z = idx / FFT_ZCHUNK, c = idx - z * FFT_ZCHUNK;
    if (c < nq) base[(long long)z * plane + q0 + c] = R[idx];
  }
}

// FP32 forward transform for a cubic N^3 grid with N known at compile time:
// the same steps as k_fft_xy_fwd<float2> and k_fft_z<2, float2>.
template <int N>
__global__ void __launch_bounds__(FFT_THREADS) k_fft_xy_fwd_ct(FftGrid g, const double* __restrict__ X, long long ldx,
                                                               float* __restrict__ S, long long lds) {
  using C = float2;
  constexpr int H = N / 2 + 1, NP = (N + 1) / 2, BUF = (NP * N > H * N) ? NP * N : H * N;
  __shared__ C twx[N];
  __shared__ C b0[BUF], b1[BUF];
  const int z = blockIdx.x, col = blockIdx.y;
  for (int t = threadIdx.x; t < N; t += blockDim.x) twx[t] = from_tw<C>(((const double2*)g.ax[0].tw)[t]);
  const double* plane = X + ldx * (long long)col + (long long)z * N * N;
  for (int idx = threadIdx.x; idx < NP * N; idx += blockDim.x) {
    const int t = idx / N, x = idx - t * N;
    const double re = plane[x + N * (2 * t)];
    const double im = (2 * t + 1 < N) ? plane[x + N * (2 * t + 1)] : 0.0;
    b0[idx] = mk<C>(to_real<float>(re), to_real<float>(im));
  }
  __syncthreads();
  C* res = fft_lines_ct<N, 1, N, -1>(b0, b1, twx, NP, 1, N);
  C* P = (res == b0) ? b1 : b0;
  for (int idx = threadIdx.x; idx < NP * H; idx += blockDim.x) {
    const int t = idx / H, k = idx - t * H;
    const C zk = res[t * N + k];
    const C zm = res[t * N + (k == 0 ? 0 : N - k)];
    P[(2 * t) * H + k] = mk<C>(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
    if (2 * t + 1 < N) P[(2 * t + 1) * H + k] = mk<C>(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
  }
  __syncthreads();
  C* other = (P == b0) ? b1 : b0;
  C* Q = fft_lines_ct<N, 1, N, -1>(P, other, twx, H, H, 1);
  C* out = (C*)(S + lds * (long long)col) + (long long)z * N * H;
  for (int idx = threadIdx.x; idx < N * H; idx += blockDim.x) out[idx] = Q[idx];
}

// ---- z pass in registers --------------------------------------------------
// Frequency held by position p of an in-place decimation-in-frequency
// transform of length n whose stages take the radices first_radix(n),
// first_radix(n / R1), ...: p = m (n / R1) + p' holds the frequency
// m + R1 freq(p') of the length n / R1 transform of sub-array m.
__host__ __device__ constexpr int dif_freq(int p, int n) {
  int f = 0, mult = 1;
  while (n > 1) {
    const int R = first_radix(n), sub = n / R;
    f += (p / sub) * mult;
    mult *= R;
    p %= sub;
    n = sub;
  }
  return f;
}

// In-place decimation-in-frequency stages on a register array: blocks of
// length L, radix R = first_radix(L), M = L / R; each R-point DFT over the
// stride-M elements of a block is followed by the twiddles W_L^(j m).
template <int N, int L, int DIR, class C>
__device__ __forceinline__ void dif_stages(C (&v)[N], const C* tw) {
  if constexpr (L > 1) {
    constexpr int R = first_radix(L), M = L / R;
#pragma unroll
    for (int b = 0; b < N / L; ++b) {
#pragma unroll
      for (int j = 0; j < M; ++j) {
        C x[R];
#pragma unroll
        for (int m = 0; m < R; ++m) x[m] = v[b * L + j + m * M];
        bfly<R, DIR>(x, tw, N);
#pragma unroll
        for (int m = 0; m < R; ++m) v[b * L + j + m * M] = (j * m == 0) ? x[m] : cmul(x[m], twid<DIR>(tw, (j * m * (N / L)) % N));
      }
    }
    dif_stages<N, M, DIR>(v, tw);
  }
}

// The z pass of the FP32 forward transform with the BF16 slices of the
// weighted spectrum out (row col of the slice matrix holds column col's
// half spectrum times the SYRK weights, 3 slices): one thread
// per z line, the whole line in registers, so there is no shared-memory
// traffic and no block barrier between the radix stages; a warp's loads and
// stores of one z row are contiguous.
constexpr int FFT_ZREG_THREADS = 128;
template <int N>
__global__ void __launch_bounds__(FFT_ZREG_THREADS) k_fft_z_slices_reg(FftGrid g, const float* S, long long lds,
                                                                      const double* __restrict__ wt,
                                                                      __nv_bfloat16* out, int rows_pad, int kp,
                                                                      int nsl) {
  using C = float2;
  constexpr int H = N / 2 + 1, PLANE = N * H;
  __shared__ C twz[N];
  for (int t = threadIdx.x; t < N; t += blockDim.x) twz[t] = from_tw<C>(((const double2*)g.ax[2].tw)[t]);
  __syncthreads();
  const int col = blockIdx.y;
  const int q = blockIdx.x * FFT_ZREG_THREADS + threadIdx.x;  // line of the x-y half plane
  if (q >= PLANE) return;
  const C* base = (const C*)(S + lds * (long long)col);
  C v[N];
#pragma unroll
  for (int z = 0; z < N; ++z) v[z] = base[(long long)z * PLANE + q];
  dif_stages<N, N, -1>(v, twz);
  const long long sstr = (long long)rows_pad * kp;
  __nv_bfloat16* o0 = out + (long long)col * kp;
#pragma unroll
  for (int p = 0; p < N; ++p) {
    const long long qq = (long long)dif_freq(p, N) * PLANE + q;
    const float w = to_real<float>(wt[qq]);
    const float vv[2] = {v[p].x * w, v[p].y * w};
    __nv_bfloat162 x0, x1, x2;
    __nv_bfloat16* p0 = reinterpret_cast<__nv_bfloat16*>(&x0);
    __nv_bfloat16* p1 = reinterpret_cast<__nv_bfloat16*>(&x1);
    __nv_bfloat16* p2 = reinterpret_cast<__nv_bfloat16*>(&x2);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      p0[h] = __float2bfloat16_rn(vv[h]);
      const float r1 = vv[h] - __bfloat162float(p0[h]);
      p1[h] = __float2bfloat16_rn(r1);
      p2[h] = __float2bfloat16_rn(r1 - __bfloat162float(p1[h]));
    }
    __nv_bfloat162* o = reinterpret_cast<__nv_bfloat162*>(o0 + 2 * qq);
    o[0] = x0;
    if (nsl > 1) o[sstr / 2] = x1;
    if (nsl > 2) o[sstr] = x2;
  }
}

// BF16 slices of w v into the row of column `col` (the common store of the
// z passes): element q of the half spectrum at out[col kp + 2 q], slices nsl.
__device__ __forceinline__ void store_spectrum_slices(float2 v, float w, __nv_bfloat16* row, long long q,
                                                      long long sstr, int nsl) {
  const float vv[2] = {v.x * w, v.y * w};
  __nv_bfloat162 x0, x1, x2;
  __nv_bfloat16* p0 = reinterpret_cast<__nv_bfloat16*>(&x0);
  __nv_bfloat16* p1 = reinterpret_cast<__nv_bfloat16*>(&x1);
  __nv_bfloat16* p2 = reinterpret_cast<__nv_bfloat16*>(&x2);
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    p0[h] = __float2bfloat16_rn(vv[h]);
    const float r1 = vv[h] - __bfloat162float(p0[h]);
    p1[h] = __float2bfloat16_rn(r1);
    p2[h] = __float2bfloat16_rn(r1 - __bfloat162float(p1[h]));
  }
  __nv_bfloat162* o = reinterpret_cast<__nv_bfloat162*>(row + 2 * q);
  o[0] = x0;
  if (nsl > 1) o[sstr / 2] = x1;
  if (nsl > 2) o[sstr] = x2;
}

// The z pass with each line split over two threads (lanes l and l + 16 of a
// warp, N even): one radix-2 decimation-in-frequency step across the pair by
// shuffles -- lane l keeps a_j + b_j, lane l + 16 keeps (a_j - b_j) W_N^j,
// a = the first half of the line, b = the second -- then a length-N/2
// transform in each thread's registers.  Lane l ends with the even
// frequencies, lane l + 16 with the odd ones.  Half the registers of
// k_fft_z_slices_reg, so twice the warps per SM to hide its latencies.
template <int N>
__global__ void __launch_bounds__(FFT_ZREG_THREADS) k_fft_z_slices_reg2(FftGrid g, const float* S, long long lds,
                                                                       const double* __restrict__ wt,
                                                                       __nv_bfloat16* out, int rows_pad, int kp,
                                                                       int nsl) {
  using C = float2;
  constexpr int H = N / 2 + 1, PLANE = N * H, HN = N / 2;
  static_assert(N % 2 == 0, "two threads per line need an even length");
  __shared__ C twz[N], tw2[HN];
  for (int t = threadIdx.x; t < N; t += blockDim.x) twz[t] = from_tw<C>(((const double2*)g.ax[2].tw)[t]);
  for (int t = threadIdx.x; t < HN; t += blockDim.x) tw2[t] = from_tw<C>(((const double2*)g.ax[2].tw)[2 * t]);
  __syncthreads();
  const int col = blockIdx.y, lane = threadIdx.x & 31, half = lane >> 4;
  const int q = blockIdx.x * (FFT_ZREG_THREADS / 2) + (threadIdx.x >> 5) * 16 + (lane & 15);
  const bool active = q < PLANE;  // every lane stays for the shuffles
  const C* base = (const C*)(S + lds * (long long)col);
  C v[HN];
#pragma unroll
  for (int j = 0; j < HN; ++j) v[j] = active ? base[(long long)(j + half * HN) * PLANE + q] : mk<C>(0.f, 0.f);
#pragma unroll
  for (int j = 0; j < HN; ++j) {
    const C o = mk<C>(__shfl_xor_sync(0xffffffffu, v[j].x, 16), __shfl_xor_sync(0xffffffffu, v[j].y, 16));
    v[j] = half == 0 ? cadd(v[j], o) : cmul(csub(o, v[j]), twid<-1>(twz, j));
  }
  dif_stages<HN, HN, -1>(v, tw2);
  if (!active) return;
  const long long sstr = (long long)rows_pad * kp;
  __nv_bfloat16* row = out + (long long)col * kp;
#pragma unroll
  for (int p = 0; p < HN; ++p) {
    const long long qq = (long long)(half + 2 * dif_freq(p, HN)) * PLANE + q;
    store_spectrum_slices(v[p], to_real<float>(wt[qq]), row, qq, sstr, nsl);
  }
}

template <int N>
static cudaError_t fft_slices_ct(const FftGrid& g, const double* X, long long ldx, int ncols, float* S32, long long lds32,
                                 const double* wt, __nv_bfloat16* out, int rows_pad, int kp, int nsl, cudaStream_t s) {
  // read theta (8 B per grid point), write nsl BF16 slices of the half spectrum
  KernelTimer kt(KF_FFT, s, (double)ncols * ((double)N * N * N * 8.0 + (double)N * N * (N / 2 + 1) * 4.0 * nsl));
  dim3 gxy(N, ncols);
  note_launch();
  k_fft_xy_fwd_ct<N><<<gxy, FFT_THREADS, 0, s>>>(g, X, ldx, S32, lds32);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  constexpr int PLANE = N * (N / 2 + 1);
  note_launch();
  if constexpr (N % 2 == 0) {
    dim3 gz((PLANE + FFT_ZREG_THREADS / 2 - 1) / (FFT_ZREG_THREADS / 2), ncols);
    k_fft_z_slices_reg2<N><<<gz, FFT_ZREG_THREADS, 0, s>>>(g, S32, lds32, wt, out, rows_pad, kp, nsl);
  } else {
    static_assert(N <= 64, "an odd compile-time length keeps its whole z line in one thread's registers");
    dim3 gz((PLANE + FFT_ZREG_THREADS - 1) / FFT_ZREG_THREADS, ncols);
    k_fft_z_slices_reg<N><<<gz, FFT_ZREG_THREADS, 0, s>>>(g, S32, lds32, wt, out, rows_pad, kp, nsl);
  }
  return cudaGetLastError();
}

size_t fft_smem_xy(const FftGrid& g) {
  int n1 = g.ax[0].n, n2 = g.ax[1].n, h = g.h;
  int npair = (n2 + 1) / 2;
  int buf = npair * n1 > h * n2 ? npair * n1 : h * n2;
  return sizeof(double2) * (size_t)(n1 + n2 + 2 * buf);
}

size_t fft_smem_z(const FftGrid& g) {
  int n3 = g.ax[2].n;
  return sizeof(double2) * (size_t)(n3 + 2 * n3 * FFT_ZCHUNK);
}

// The FP32 kernels use half of these byte counts.

// The limit is an attribute of the kernel (per device), shared by every
// context: it only ever grows, so that a context on a smaller grid created
// later does not lower it below what an existing context launches with.
cudaError_t fft_configure(size_t smem_xy, size_t smem_z) {
  static std::mutex mu;
  static size_t cur_xy[64] = {}, cur_z[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (smem_xy > cur_xy[dev]) {
    e = cudaFuncSetAttribute(k_fft_xy_fwd<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_xy);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_fft_xy_fwd<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_xy);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_fft_xy_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_xy);
    if (e != cudaSuccess) return e;
    cur_xy[dev] = smem_xy;
  }
  if (smem_z > cur_z[dev]) {
    e = cudaFuncSetAttribute(k_fft_z<0, double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_z);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_fft_z<2, float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_z);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_fft_z<1, double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_z);
    if (e != cudaSuccess) return e;
    cur_z[dev] = smem_z;
  }
  return cudaSuccess;
}

cudaError_t launch_fft_forward(const FftGrid& g, const double* X, long long ldx, int ncols, double* S,
                               long long lds, const double* wt, size_t smem_xy, size_t smem_z,
                               cudaStream_t s) {
  if (ncols <= 0) return cudaSuccess;
  const double nr = (double)g.ax[0].n * g.ax[1].n * g.ax[2].n, nh = (double)g.h * g.ax[1].n * g.ax[2].n;
  KernelTimer kt(KF_FFT, s, ncols * (nr * 8.0 + nh * 16.0));  // read X, write the half spectrum
  dim3 gxy(g.ax[2].n, ncols);
  note_launch();
  k_fft_xy_fwd<double2><<<gxy, FFT_THREADS, smem_xy, s>>>(g, X, ldx, S, lds);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int plane = g.ax[1].n * g.h;
  dim3 gz((plane + FFT_ZCHUNK - 1) / FFT_ZCHUNK, ncols);
  note_launch();
  k_fft_z<0, double2><<<gz, FFT_THREADS, smem_z, s>>>(g, S, lds, wt, nullptr, 0, 0, 0);
  return cudaGetLastError();
}

cudaError_t launch_fft_convolve(const FftGrid& g, const double* In, long long ldin, int ncols, double* S,
                                long long lds, const double* wt, const double* Add, long long ldadd,
                                double* Y, long long ldy, size_t smem_xy, size_t smem_z,
                                cudaStream_t s) {
  if (ncols <= 0) return cudaSuccess;
  const double nr = (double)g.ax[0].n * g.ax[1].n * g.ax[2].n;
  KernelTimer kt(KF_FFT, s, ncols * nr * 8.0 * (Add ? 3.0 : 2.0));  // read In (and Add), write Y
  dim3 gxy(g.ax[2].n, ncols);
  note_launch();
  k_fft_xy_fwd<double2><<<gxy, FFT_THREADS, smem_xy, s>>>(g, In, ldin, S, lds);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int plane = g.ax[1].n * g.h;
  dim3 gz((plane + FFT_ZCHUNK - 1) / FFT_ZCHUNK, ncols);
  note_launch();
  k_fft_z<1, double2><<<gz, FFT_THREADS, smem_z, s>>>(g, S, lds, wt, nullptr, 0, 0, 0);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  note_launch();
  k_fft_xy_inv<<<gxy, FFT_THREADS, smem_xy, s>>>(g, S, lds, Add, ldadd, Y, ldy);
  return cudaGetLastError();
}

}  // namespace isdf

namespace isdf {

cudaError_t launch_fft_forward_slices(const FftGrid& g, const double* X, long long ldx, int ncols, float* S32,
                                      long long lds32, const double* wt, __nv_bfloat16* out, int rows_pad, int kp,
                                      int nsl, size_t smem_xy, size_t smem_z, cudaStream_t s) {
  if (ncols <= 0) return cudaSuccess;
  const int n = g.ax[0].n;
  // bf16x2 stores of (re, im) need kp and rows_pad * kp even: kp is a multiple of 64
  if (n == g.ax[1].n && n == g.ax[2].n && (kp % 2) == 0) {
    switch (n) {
#define ISDF_FFT_CT(N) \
  case N: return fft_slices_ct<N>(g, X, ldx, ncols, S32, lds32, wt, out, rows_pad, kp, nsl, s);
      ISDF_FFT_CT(16) ISDF_FFT_CT(24) ISDF_FFT_CT(27) ISDF_FFT_CT(30) ISDF_FFT_CT(32) ISDF_FFT_CT(36)
      ISDF_FFT_CT(40) ISDF_FFT_CT(45) ISDF_FFT_CT(48) ISDF_FFT_CT(50) ISDF_FFT_CT(54) ISDF_FFT_CT(60)
      ISDF_FFT_CT(64) ISDF_FFT_CT(72)
#undef ISDF_FFT_CT
      default: break;
    }
  }
  const double nr = (double)g.ax[0].n * g.ax[1].n * g.ax[2].n, nh = (double)g.h * g.ax[1].n * g.ax[2].n;
  KernelTimer kt(KF_FFT, s, ncols * (nr * 8.0 + nh * 4.0 * nsl));
  dim3 gxy(g.ax[2].n, ncols);
  note_launch();
  k_fft_xy_fwd<float2><<<gxy, FFT_THREADS, smem_xy / 2, s>>>(g, X, ldx, S32, lds32);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int plane = g.ax[1].n * g.h;
  dim3 gz((plane + FFT_ZCHUNK - 1) / FFT_ZCHUNK, ncols);
  note_launch();
  k_fft_z<2, float2><<<gz, FFT_THREADS, smem_z / 2, s>>>(g, S32, lds32, wt, out, rows_pad, kp, nsl);
  return cudaGetLastError();
}

}  // namespace isdf
