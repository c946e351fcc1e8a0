// Mixed-path CholQR factor (Sec. "Ground-state solution": orthonormalisation of the block by
// the Cholesky factor of its overlap S = Psi^H Psi, Psi <- Psi L^{-H}).
//
// The FP64 factorisation of an n <= 160 matrix in one CTA is bound by GB300's FP64 rate, so
// the factor is refined in two FP32 passes instead (the two-pass idea of CholeskyQR2,
// applied to the small factor only):
//
//   1. L1 L1^H = S       FP32 Cholesky in shared memory, M1 = L1^{-1}        (one CTA)
//   2. S2 = M1 S M1^H    FP64 triangular products, S2 = I + O(eps_32 kappa)   (many CTAs)
//   3. L2 L2^H = S2      FP32 Cholesky, M2 = L2^{-1}                          (one CTA)
//   4. M = conj(M2 M1)   FP64, lower triangular                               (many CTAs)
//
// L1 L2 is lower triangular with a positive diagonal and (L1 L2)(L1 L2)^H = S, so M2 M1 is
// the inverse of S's Cholesky factor; pass 3 factors a matrix within eps_32 kappa(S) of the
// identity, so M carries ~eps_32 relative error, which the 24-bit rotation cannot resolve
// anyway.  A pivot <= tol * S_jj in either pass sets status = j + 1 and M = I.
#include "kernels.h"

namespace ks {

namespace {

constexpr int C32_MAXN = 160;
constexpr int C32_THREADS = 1024;

// Column-major packed lower triangle: element (r, c), r >= c, at coff(c) + r - c.
__device__ __forceinline__ int coff(int c, int n) { return c * n - (c * (c - 1)) / 2; }

// One CTA.  Reads the lower triangle of S (n x n, row-major), writes X = L^{-1} (lower,
// zeros above; conj(X) when conj_out) to Out.  Both loops are right-looking with the
// column scaling deferred, so each step is one barrier:
//   Cholesky: U_ik -= U_ij conj(U_kj) / d_j  (U_jj = d_j, L_ij = U_ij / sqrt(d_j))
//   inverse:  W = U^{-1} row by row, Y_r -= U_ri Y_i / d_i, then X_ic = Y_ic / sqrt(d_i).
// Work mapping: warps over columns, lanes over rows (unit stride in the packed layout).
__global__ void __launch_bounds__(C32_THREADS, 1)
    k_chol32_inverse(const double2* __restrict__ S, int n, double tol, int conj_out, int* __restrict__ status,
                     double2* __restrict__ Out) {
  extern __shared__ float2 c32[];
  const int npk = n * (n + 1) / 2;
  float2* U = c32;          // factor, unscaled columns
  float2* Y = c32 + npk;    // inverse, unscaled rows
  __shared__ float dg[C32_MAXN], sjj[C32_MAXN];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  constexpr int NW = C32_THREADS / 32;

  for (int c = warp; c < n; c += NW)
    for (int r = c + lane; r < n; r += 32) {
      const double2 v = S[(size_t)r * n + c];
      U[coff(c, n) + r - c] = make_float2((float)v.x, r == c ? 0.f : (float)v.y);
      Y[coff(c, n) + r - c] = make_float2(r == c ? 1.f : 0.f, 0.f);
    }
  for (int j = t; j < n; j += C32_THREADS) sjj[j] = (float)S[(size_t)j * n + j].x;
  __syncthreads();

  int bad = 0;
  for (int j = 0; j < n; ++j) {
    const float d = U[coff(j, n)].x;                    // every thread reads the same pivot
    if (!(d > (float)tol * sjj[j]) || !isfinite(d)) {
      bad = j + 1;
      break;
    }
    if (t == 0) dg[j] = d;
    const float inv = 1.f / d;
    const float2* colj = U + coff(j, n) - j;            // colj[r] = U_rj
    for (int k = j + 1 + warp; k < n; k += NW) {
      const float2 b = colj[k];
      const float2 bs = make_float2(b.x * inv, -b.y * inv);   // conj(U_kj) / d_j
      float2* colk = U + coff(k, n) - k;
      for (int i = k + lane; i < n; i += 32) {
        const float2 a = colj[i];
        float2 v = colk[i];
        v.x -= a.x * bs.x - a.y * bs.y;
        v.y -= a.x * bs.y + a.y * bs.x;
        colk[i] = v;
      }
    }
    __syncthreads();
  }
  if (bad) {
    for (int e = t; e < n * n; e += C32_THREADS) Out[e] = make_double2((e / n == e % n) ? 1.0 : 0.0, 0.0);
    if (t == 0) atomicCAS(status, 0, bad);
    return;
  }
  // Y = U^{-1} D (rows unscaled): for each i, rows r > i lose U_ri Y_i / d_i
  for (int i = 0; i + 1 < n; ++i) {
    const float inv = 1.f / dg[i];
    const float2* coli = U + coff(i, n) - i;            // coli[r] = U_ri
    for (int c = warp; c <= i; c += NW) {
      float2* ycol = Y + coff(c, n) - c;                 // ycol[r] = Y_rc
      const float2 yi = ycol[i];
      const float2 ys = make_float2(yi.x * inv, yi.y * inv);
      for (int r = i + 1 + lane; r < n; r += 32) {
        const float2 u = coli[r];
        float2 v = ycol[r];
        v.x -= u.x * ys.x - u.y * ys.y;
        v.y -= u.x * ys.y + u.y * ys.x;
        ycol[r] = v;
      }
    }
    __syncthreads();
  }
  // X_rc = Y_rc / sqrt(d_r)
  const float sgn = conj_out ? -1.f : 1.f;
  for (int e = t; e < n * n; e += C32_THREADS) {
    const int r = e / n, c = e - (e / n) * n;
    if (c <= r) {
      const float2 y = Y[coff(c, n) + r - c];
      const float sc = rsqrtf(dg[r]);
      Out[e] = make_double2((double)(y.x * sc), (double)(sgn * y.y * sc));
    } else {
      Out[e] = make_double2(0.0, 0.0);
    }
  }
}

// FP64 triangular products on 8 x 8 output tiles, one output per thread:
//   MODE 0: C = S M^H            C_ij = sum_{k <= j} S_ik conj(M_jk)          (all tiles)
//   MODE 1: C = M T (lower part)  C_ij = sum_{k <= i} M_ik T_kj, i >= j
//   MODE 2: C = conj(A B)         C_ij = conj(sum_{j <= k <= i} A_ik B_kj), i >= j; 0 above;
//           C = I once *status is set
template <int MODE>
__global__ void __launch_bounds__(64) k_tri_product(const double2* __restrict__ A, const double2* __restrict__ B,
                                                    int n, const int* __restrict__ status, double2* __restrict__ C) {
  const int i = blockIdx.y * 8 + (threadIdx.x >> 3), j = blockIdx.x * 8 + (threadIdx.x & 7);
  if (MODE == 2 && *status != 0) {
    if (i < n && j < n) C[(size_t)i * n + j] = make_double2(i == j ? 1.0 : 0.0, 0.0);
    return;
  }
  if (MODE != 0 && blockIdx.x > blockIdx.y) {           // strictly upper tile
    if (MODE == 2 && i < n && j < n) C[(size_t)i * n + j] = make_double2(0.0, 0.0);
    return;
  }
  if (i >= n || j >= n) return;
  double re = 0.0, im = 0.0;
  if (MODE == 0) {
    for (int k = 0; k <= j; ++k) {
      const double2 a = A[(size_t)i * n + k], b = B[(size_t)j * n + k];
      re += a.x * b.x + a.y * b.y;
      im += a.y * b.x - a.x * b.y;
    }
    C[(size_t)i * n + j] = make_double2(re, im);
  } else if (MODE == 1) {
    if (j > i) return;
    for (int k = 0; k <= i; ++k) {
      const double2 a = A[(size_t)i * n + k], b = B[(size_t)k * n + j];
      re += a.x * b.x - a.y * b.y;
      im += a.x * b.y + a.y * b.x;
    }
    C[(size_t)i * n + j] = make_double2(re, im);
  } else {
    if (j > i) {
      C[(size_t)i * n + j] = make_double2(0.0, 0.0);
      return;
    }
    for (int k = j; k <= i; ++k) {
      const double2 a = A[(size_t)i * n + k], b = B[(size_t)k * n + j];
      re += a.x * b.x - a.y * b.y;
      im += a.x * b.y + a.y * b.x;
    }
    C[(size_t)i * n + j] = make_double2(re, -im);
  }
}

}  // namespace

size_t cholesky_mixed_workspace(int n) { return (size_t)3 * n * n; }

void cholesky_inverse_mixed(const double2* S, double2* M, int n, double tol, double2* work, int* status,
                            cudaStream_t s) {
  if (n > C32_MAXN) fail(KS_ERR_ARG, "cholesky_inverse_mixed: n=%d > %d", n, C32_MAXN);
  const size_t smem = (size_t)n * (n + 1) * sizeof(float2);
  static bool attr_set = false;
  if (!attr_set) {
    KS_CUDA(cudaFuncSetAttribute(k_chol32_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)((size_t)C32_MAXN * (C32_MAXN + 1) * sizeof(float2))));
    attr_set = true;
  }
  double2* M1 = work;
  double2* T = work + (size_t)n * n;
  double2* M2 = work + (size_t)2 * n * n;
  const int nt = (n + 7) / 8;
  const dim3 grid(nt, nt);
  k_chol32_inverse<<<1, C32_THREADS, smem, s>>>(S, n, tol, 0, status, M1);
  KS_CHECK_LAUNCH();
  k_tri_product<0><<<grid, 64, 0, s>>>(S, M1, n, status, T);
  KS_CHECK_LAUNCH();
  k_tri_product<1><<<grid, 64, 0, s>>>(M1, T, n, status, M2);      // S2 (lower) into M2's storage
  KS_CHECK_LAUNCH();
  k_chol32_inverse<<<1, C32_THREADS, smem, s>>>(M2, n, tol, 0, status, T);
  KS_CHECK_LAUNCH();
  k_tri_product<2><<<grid, 64, 0, s>>>(T, M1, n, status, M);
  KS_CHECK_LAUNCH();
}

}  // namespace ks
