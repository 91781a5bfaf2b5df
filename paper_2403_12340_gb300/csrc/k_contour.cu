// Contour-integral polarizability (Algorithm 2): -2 B = -2 C Omega^-1 C^T
// without the sum over pairs.
//
// With a closed contour that encloses the unoccupied energies and none of
// the occupied ones, 1/(e_v - e_c) = -(1/2 pi i) oint dl / ((l - e_v)(l - e_c)),
// so B = -(1/2 pi i) oint J(l) dl with the Hadamard product
//   J(l) = (Psi_v diag(1/(l - e_v)) Psi_v^T) .* (Psi_c diag(1/(l - e_c)) Psi_c^T)
// of two resolvent Grams at the interpolation points.  Real orbitals make J
// conjugate-symmetric, so B = (1/pi) Im of the integral over the upper half
// of the contour, taken along the image of t in [-K + i K'/2, K + i K'/2]
// under z(t) = e_N + sqrt(q Q) (1/k + sn(t, k)) / (1/k - sn(t, k)) (the map of
// Algorithm 2: q the gap, Q the width from the highest occupied energy e_N to
// the top of the unoccupied band, k = (sqrt(Q/q) - 1) / (sqrt(Q/q) + 1));
// that image runs left to right, which is why the sign is +.  The midpoint
// rule in t converges geometrically (Eq. rel_err_Cauchy).
//
// Cost: per node 2 r^2 N_e FP64 flops for the two complex resolvent Grams
// (lower tiles), against r^2 N_v N_c for the pair sum: the contour wins when
// N_v N_c > 2 N_nodes N_e.
#include <cmath>
#include <complex>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace isdf {

namespace {

// ---- host: complete elliptic integral and Jacobi functions ----------------
double ellip_k(double k) {  // K(k) = pi / (2 agm(1, k'))
  double a = 1.0, b = std::sqrt(1.0 - k * k);
  for (int i = 0; i < 60 && std::fabs(a - b) > 1e-16 * a; ++i) {
    const double an = 0.5 * (a + b);
    b = std::sqrt(a * b);
    a = an;
  }
  return M_PI / (a + b);
}

// sn, cn, dn of a real argument by the descending Landen (AGM) recursion
void jacobi(double u, double k, double& sn, double& cn, double& dn) {
  double a[48], c[48];
  a[0] = 1.0;
  c[0] = k;
  double b = std::sqrt(1.0 - k * k);
  int n = 0;
  while (std::fabs(c[n]) > 1e-17 && n < 46) {
    a[n + 1] = 0.5 * (a[n] + b);
    c[n + 1] = 0.5 * (a[n] - b);
    b = std::sqrt(a[n] * b);
    ++n;
  }
  double phi = std::ldexp(a[n] * u, n), prev = phi;
  for (int i = n; i > 0; --i) {
    prev = phi;
    phi = 0.5 * (phi + std::asin(c[i] * std::sin(phi) / a[i]));
  }
  sn = std::sin(phi);
  cn = std::cos(phi);
  dn = n > 0 ? cn / std::cos(prev - phi) : 1.0;
}

__global__ void __launch_bounds__(256) k_contour_polar(const double* __restrict__ phimu, long long ldp, int r, int n_v,
                                                     int n_e, const double2* __restrict__ wtab,
                                                     const double2* __restrict__ wnode, int nodes_per_split,
                                                     int n_nodes, double scale, double* D, long long ldd,
                                                     double* partial) {
  constexpr int BT = 32, BK = 64;
  __shared__ double As[BK][BT + 1], Bs[BK][BT + 1];
  __shared__ double2 Ws[BK];
  int mt, nt;
  lower_tile(blockIdx.x, mt, nt);
  const int m0 = mt * BT, n0 = nt * BT;
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  const int j0 = blockIdx.z * nodes_per_split;
  const int j1 = min(n_nodes, j0 + nodes_per_split);
  double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  for (int j = j0; j < j1; ++j) {
    double vr[2][2] = {{0, 0}, {0, 0}}, vi[2][2] = {{0, 0}, {0, 0}};
    double cr[2][2] = {{0, 0}, {0, 0}}, ci[2][2] = {{0, 0}, {0, 0}};
    for (int k0 = 0; k0 < n_e; k0 += BK) {
      for (int idx = t; idx < BK * BT; idx += 256) {
        const int row = idx % BT, kk = idx / BT, k = k0 + kk;
        As[kk][row] = (m0 + row < r && k < n_e) ? phimu[(m0 + row) + ldp * (long long)k] : 0.0;
        Bs[kk][row] = (n0 + row < r && k < n_e) ? phimu[(n0 + row) + ldp * (long long)k] : 0.0;
      }
      if (t < BK) Ws[t] = (k0 + t < n_e) ? wtab[(long long)j * n_e + k0 + t] : make_double2(0.0, 0.0);
      __syncthreads();
      const int kend = min(BK, n_e - k0);
      const int kv = max(0, min(kend, n_v - k0));  // chunk entries [0, kv) are occupied orbitals
      for (int kk = 0; kk < kv; ++kk) {
        const double2 w = Ws[kk];
        const double a0 = As[kk][tx], a1 = As[kk][tx + 16], b0 = Bs[kk][ty], b1 = Bs[kk][ty + 16];
        const double r0 = a0 * w.x, r1 = a1 * w.x, i0 = a0 * w.y, i1 = a1 * w.y;
        vr[0][0] = fma(r0, b0, vr[0][0]); vr[0][1] = fma(r0, b1, vr[0][1]);
        vr[1][0] = fma(r1, b0, vr[1][0]); vr[1][1] = fma(r1, b1, vr[1][1]);
        vi[0][0] = fma(i0, b0, vi[0][0]); vi[0][1] = fma(i0, b1, vi[0][1]);
        vi[1][0] = fma(i1, b0, vi[1][0]); vi[1][1] = fma(i1, b1, vi[1][1]);
      }
      for (int kk = kv; kk < kend; ++kk) {
        const double2 w = Ws[kk];
        const double a0 = As[kk][tx], a1 = As[kk][tx + 16], b0 = Bs[kk][ty], b1 = Bs[kk][ty + 16];
        const double r0 = a0 * w.x, r1 = a1 * w.x, i0 = a0 * w.y, i1 = a1 * w.y;
        cr[0][0] = fma(r0, b0, cr[0][0]); cr[0][1] = fma(r0, b1, cr[0][1]);
        cr[1][0] = fma(r1, b0, cr[1][0]); cr[1][1] = fma(r1, b1, cr[1][1]);
        ci[0][0] = fma(i0, b0, ci[0][0]); ci[0][1] = fma(i0, b1, ci[0][1]);
        ci[1][0] = fma(i1, b0, ci[1][0]); ci[1][1] = fma(i1, b1, ci[1][1]);
      }
      __syncthreads();
    }
    // acc += Im(J w_node), J = (vr + i vi) .* (cr + i ci)
    const double2 wn = wnode[j];
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const double jr = vr[p][q] * cr[p][q] - vi[p][q] * ci[p][q];
        const double ji = vr[p][q] * ci[p][q] + vi[p][q] * cr[p][q];
        acc[p][q] += jr * wn.y + ji * wn.x;
      }
  }
#pragma unroll
  for (int p = 0; p < 2; ++p)
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int m = m0 + tx + 16 * p, n = n0 + ty + 16 * q;
      if (m >= r || n >= r) continue;
      const double v = scale * acc[p][q];
      if (partial) {
        partial[(long long)blockIdx.z * r * r + m + (long long)r * n] = v;
      } else {
        D[m + ldd * n] = v;
        if (mt != nt) D[n + ldd * m] = v;
      }
    }
}

}  // namespace

int contour_nodes_recommended(double gap, double width, double tol) {
  // Eq. rel_err_Cauchy: error ~ exp(-pi^2 N / (2 log(Q/q) + 6))
  const double n = std::log(1.0 / tol) * (2.0 * std::log(width / gap) + 6.0) / (M_PI * M_PI);
  return (int)std::ceil(n);
}

cudaError_t contour_tables(const double* energies, int n_v, int n_c, int n_nodes, std::vector<double>& wtab,
                           std::vector<double>& wnode) {
  const int n_e = n_v + n_c;
  double e_n = energies[0], e_lo = energies[n_v], e_hi = energies[n_v];
  for (int i = 0; i < n_v; ++i) e_n = std::max(e_n, energies[i]);
  for (int i = n_v; i < n_e; ++i) {
    e_lo = std::min(e_lo, energies[i]);
    e_hi = std::max(e_hi, energies[i]);
  }
  const double q = e_lo - e_n, big_q = e_hi - e_n;
  if (!(q > 0.0) || n_nodes < 1) return cudaErrorInvalidValue;
  const double ratio = std::sqrt(big_q / q);
  // a flat unoccupied band (Q = q) degenerates the map; a slightly wider one is exact as well
  const double k = std::max((ratio - 1.0) / (ratio + 1.0), 1e-6);
  const double kk = ellip_k(k), kkp = ellip_k(std::sqrt(1.0 - k * k));
  const double scale = std::sqrt(q * big_q), h = 2.0 * kk / n_nodes, kp = std::sqrt(1.0 - k * k);
  wtab.assign((size_t)2 * n_nodes * n_e, 0.0);
  wnode.assign((size_t)2 * n_nodes, 0.0);
  double s1, c1, d1;
  jacobi(0.5 * kkp, kp, s1, c1, d1);
  for (int j = 0; j < n_nodes; ++j) {
    double s, c, d;
    jacobi(-kk + (j + 0.5) * h, k, s, c, d);
    const double den = c1 * c1 + k * k * s * s * s1 * s1;
    const std::complex<double> sn(s * d1 / den, c * d * s1 * c1 / den);
    const std::complex<double> cn(c * c1 / den, -s * d * s1 * d1 / den);
    const std::complex<double> dn(d * c1 * d1 / den, -k * k * s * c * s1 / den);
    const std::complex<double> z = e_n + scale * (1.0 / k + sn) / (1.0 / k - sn);
    const std::complex<double> w = h * scale * (2.0 / k) * cn * dn / ((1.0 / k - sn) * (1.0 / k - sn));
    wnode[2 * j] = w.real();
    wnode[2 * j + 1] = w.imag();
    for (int i = 0; i < n_e; ++i) {
      const std::complex<double> rv = 1.0 / (z - energies[i]);
      wtab[2 * ((size_t)j * n_e + i)] = rv.real();
      wtab[2 * ((size_t)j * n_e + i) + 1] = rv.imag();
    }
  }
  return cudaSuccess;
}

cudaError_t launch_contour_polarizability(const double* phimu, long long ldp, int r, int n_v, int n_c,
                                          const double* d_wtab, const double* d_wnode, int n_nodes, double* D,
                                          long long ldd, double* partial, size_t partial_cap, int num_sms,
                                          cudaStream_t s) {
  if (r <= 0) return cudaSuccess;
  const int n_e = n_v + n_c;
  const int tm = (r + 31) / 32;
  const long long tiles = (long long)tm * (tm + 1) / 2;
  int split = (int)std::min<long long>(n_nodes, (2LL * num_sms + tiles - 1) / tiles);
  if (split < 1) split = 1;
  while (split > 1 && (size_t)split * r * r > partial_cap) --split;
  const int per = (n_nodes + split - 1) / split;
  split = (n_nodes + per - 1) / per;
  dim3 grid((unsigned)tiles, 1, split);
  cudaError_t e;
  {
    KernelTimer kt(KF_FP64_GEMM, s, 2.0 * n_nodes * (double)r * (r + 1) * n_e);
    note_launch();
    k_contour_polar<<<grid, 256, 0, s>>>(phimu, ldp, r, n_v, n_e, reinterpret_cast<const double2*>(d_wtab),
                                         reinterpret_cast<const double2*>(d_wnode), per, n_nodes, -2.0 / M_PI, D,
                                         ldd, split > 1 ? partial : nullptr);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess || split == 1) return e;
  return launch_splitk_reduce(partial, split, r, r, 1.0, 0.0, D, ldd, true, 32, s);
}

}  // namespace isdf
