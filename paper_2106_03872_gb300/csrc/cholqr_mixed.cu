// Mixed-path CholQR factor (Sec. "Ground-state solution": orthonormalisation of the block by
// the Cholesky factor of its overlap S = Psi^H Psi, Psi <- Psi L^{-H}).
//
// The FP64 factorisation of an n <= 160 matrix in one CTA is bound by GB300's FP64 rate, so
// the factor comes from one FP32 pass refined in FP64:
//
//   1. L1 L1^H = S       FP32 Cholesky in shared memory, M1 = L1^{-1}        (one CTA)
//   2. S2 = M1 S M1^H    FP64 triangular products, S2 = I + E with |E| ~ eps_32 kappa(S)
//   3. M = conj((I - Phi(E)) M1), Phi(E) = strictly lower part of E plus half its diagonal
//
// (I + Phi(E)) is the Cholesky factor of I + E to first order, so (I - Phi(E)) M1 is the
// inverse Cholesky factor of S up to O(E^2) ~ (eps_32 kappa(S))^2 -- below the 24-bit
// precision of the states for kappa(S) up to ~1e4.  A pivot <= tol * S_jj sets status = j + 1
// and M = I.
//
// Without refinement the result is M1 itself (conjugated), accurate to ~eps_32 kappa(S)
// sqrt(n).  The pipelined block iteration takes that form: it uses only the FP32 copy of M,
// whose rounding is of the order of the refinement's correction for the well-conditioned S of
// an iterate, and the next iteration's CholQR starts again from the S of the new block.
#include <type_traits>

#include "kernels.h"

namespace ks {

namespace {

constexpr int C32_MAXN = 160;          // square array in shared memory
constexpr int C32_MAXN_GLOBAL = 256;   // square array in global memory
constexpr int C32_THREADS = 1024;

// One CTA.  Reads the lower triangle of S (n x n, row-major), writes X = L^{-1} (lower,
// zeros above; conj(X) when conj_out) to Out, and an FP32 copy to Out32 when it is given.
//
// Shared memory holds one square [n][ld] array: L_rc (r >= c) at [c][r] (column-major, so
// lanes running along a column touch consecutive words) and X_rc (r > c) at [r][c], i.e. in
// the unused upper triangle; X's diagonal is a separate vector.  Blocked by CB columns, each
// block step three barriers:
//   (a) warp 0 factors the diagonal block in registers (lane = row, the pivot column is
//       broadcast by shuffles) and inverts it in registers;
//   (b) panel L_iJ = A_iJ W_J^H for the rows below (all threads);
//   (c) trailing update A_ik -= sum_{c in J} L_ic conj(L_kc) (warps over columns k, lanes
//       over rows i; conj(L_kJ) held in registers).
// Then the off-diagonal blocks of X by block rows I: T_IJ = sum_{K=J}^{I-1} L_IK X_KJ,
// X_IJ = -W_I T_IJ for all J < I at once.
constexpr int CB = 8;

__device__ __forceinline__ float2 c_mul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ float2 c_mulc(float2 a, float2 b) {   // a * conj(b)
  return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ float2 shfl2(float2 v, int src) {
  return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

// MAXN: the largest n; GLB: the square array lives in global memory (gU, n (n + 1) values,
// L2-resident) instead of shared memory, for n beyond what shared memory holds (160 < n <= 256).
template <int MAXN, bool GLB>
__global__ void __launch_bounds__(C32_THREADS, 1)
    k_chol32_inverse(const double2* __restrict__ S, int n, double tol, int conj_out, int* __restrict__ status,
                     double2* __restrict__ Out, float2* __restrict__ Out32, float2* __restrict__ gU) {
  extern __shared__ float2 c32[];
  const int ld = n + 1;
  float2* U = GLB ? gU : c32;
  __shared__ float sjj[MAXN];
  __shared__ float2 xd[MAXN];                                        // diagonal of X
  __shared__ int s_bad;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  constexpr int NW = C32_THREADS / 32;
#define UL(r, c) U[(c) * ld + (r)]
#define XU(r, c) U[(r) * ld + (c)]
#define XL(r, c) ((r) == (c) ? xd[r] : XU(r, c))

  for (int e = t; e < n * n; e += C32_THREADS) {
    const int r = e / n, c = e - (e / n) * n;
    if (c <= r) {
      const double2 v = S[e];
      UL(r, c) = make_float2((float)v.x, r == c ? 0.f : (float)v.y);
    }
  }
  for (int j = t; j < n; j += C32_THREADS) sjj[j] = (float)S[(size_t)j * n + j].x;
  if (t == 0) s_bad = 0;
  __syncthreads();

  for (int J = 0; J < n; J += CB) {
    const int jb = min(CB, n - J), J1 = J + jb;
    // (a) diagonal block in warp 0's registers: lane r holds row J + r
    if (warp == 0) {
      float2 a[CB];
#pragma unroll
      for (int c = 0; c < CB; ++c) a[c] = (c <= lane && lane < jb) ? UL(J + lane, J + c) : make_float2(0.f, 0.f);
      int bad = 0;
#pragma unroll
      for (int j = 0; j < CB; ++j) {
        if (j < jb && !bad) {
          const float d = __shfl_sync(0xffffffffu, a[j].x, j);
          if (!(d > (float)tol * sjj[J + j]) || !isfinite(d)) {
            bad = J + j + 1;
          } else {
            const float ljj = sqrtf(d), inv = 1.f / ljj;
            if (lane == j) a[j] = make_float2(ljj, 0.f);
            else if (lane > j) a[j] = make_float2(a[j].x * inv, a[j].y * inv);
#pragma unroll
            for (int k = j + 1; k < CB; ++k) {
              const float2 lkj = shfl2(a[j], k);
              if (k <= lane) {
                const float2 p = c_mulc(a[j], lkj);
                a[k].x -= p.x;
                a[k].y -= p.y;
              }
            }
          }
        }
      }
      if (bad) {
        if (lane == 0) s_bad = bad;
      } else {
#pragma unroll
        for (int c = 0; c < CB; ++c)
          if (c <= lane && lane < jb) UL(J + lane, J + c) = a[c];
        // W = L_JJ^{-1} by rows: row j final after division by L_jj, rows r > j lose L_rj W_j
        float2 w[CB];
#pragma unroll
        for (int c = 0; c < CB; ++c) w[c] = make_float2(c == lane ? 1.f : 0.f, 0.f);
#pragma unroll
        for (int j = 0; j < CB; ++j) {
          if (j < jb) {
            const float ij = 1.f / __shfl_sync(0xffffffffu, a[j].x, j);
            if (lane == j) {
#pragma unroll
              for (int c = 0; c <= j; ++c) w[c] = make_float2(w[c].x * ij, w[c].y * ij);
            }
#pragma unroll
            for (int c = 0; c <= j; ++c) {
              const float2 wj = shfl2(w[c], j);
              if (lane > j) {
                const float2 p = c_mul(a[j], wj);
                w[c].x -= p.x;
                w[c].y -= p.y;
              }
            }
          }
        }
        if (lane < jb) {
#pragma unroll
          for (int c = 0; c < CB; ++c) {
            if (c < lane) XU(J + lane, J + c) = w[c];
            else if (c == lane) xd[J + lane] = w[c];
          }
        }
      }
    }
    __syncthreads();
    if (s_bad) break;                                                // uniform
    const int rows = n - J1;
    if (rows == 0) break;
    // (b) panel: L_ic = sum_{k=J}^{c} A_ik conj(W_ck); lanes run along i
    float2 pv[(MAXN * CB + C32_THREADS - 1) / C32_THREADS];
#pragma unroll
    for (int q = 0; q < (MAXN * CB + C32_THREADS - 1) / C32_THREADS; ++q) {
      const int idx = t + q * C32_THREADS;
      pv[q] = make_float2(0.f, 0.f);
      if (idx < rows * jb) {
        const int i = J1 + idx % rows, c = J + idx / rows;
        for (int k = J; k <= c; ++k) {
          const float2 p = c_mulc(UL(i, k), XL(c, k));
          pv[q].x += p.x;
          pv[q].y += p.y;
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < (MAXN * CB + C32_THREADS - 1) / C32_THREADS; ++q) {
      const int idx = t + q * C32_THREADS;
      if (idx < rows * jb) UL(J1 + idx % rows, J + idx / rows) = pv[q];
    }
    __syncthreads();
    // (c) trailing update, columns k >= J1
    for (int k = J1 + warp; k < n; k += NW) {
      float2 lk[CB];
#pragma unroll
      for (int c = 0; c < CB; ++c) {
        const float2 v = c < jb ? UL(k, J + c) : make_float2(0.f, 0.f);
        lk[c] = make_float2(v.x, -v.y);
      }
      for (int i = k + lane; i < n; i += 32) {
        float2 acc = make_float2(0.f, 0.f);
        const float2* col = U + J * ld + i;                          // col[c * ld] = L_{i, J+c}
#pragma unroll
        for (int c = 0; c < CB; ++c) {
          if (c < jb) {
            const float2 p = c_mul(col[c * ld], lk[c]);
            acc.x += p.x;
            acc.y += p.y;
          }
        }
        const float2 v = UL(i, k);
        UL(i, k) = make_float2(v.x - acc.x, v.y - acc.y);
      }
    }
    __syncthreads();
  }
  if (s_bad) {
    for (int e = t; e < n * n; e += C32_THREADS) {
      const bool diag = e / n == e % n;
      Out[e] = make_double2(diag ? 1.0 : 0.0, 0.0);
      if (Out32) Out32[e] = make_float2(diag ? 1.f : 0.f, 0.f);
    }
    if (t == 0) atomicCAS(status, 0, s_bad);
    return;
  }
  // off-diagonal blocks of X, block row by block row
  for (int I0 = CB; I0 < n; I0 += CB) {
    const int ib = min(CB, n - I0);
    // T_rc = sum_{k=c}^{I0-1} L_rk X_kc into X(r, c), r in block row I, c < I0 (lanes along r)
    for (int idx = t; idx < ib * I0; idx += C32_THREADS) {
      const int r = I0 + idx % ib, c = idx / ib;
      float2 acc = c_mul(UL(r, c), xd[c]);
      for (int k = c + 1; k < I0; ++k) {
        const float2 p = c_mul(UL(r, k), XU(k, c));
        acc.x += p.x;
        acc.y += p.y;
      }
      XU(r, c) = acc;
    }
    __syncthreads();
    // X_rc = -sum_{r'=I0}^{r} W_I[r][r'] T_r'c
    float2 xv[(CB * MAXN + C32_THREADS - 1) / C32_THREADS];
#pragma unroll
    for (int q = 0; q < (CB * MAXN + C32_THREADS - 1) / C32_THREADS; ++q) {
      const int idx = t + q * C32_THREADS;
      xv[q] = make_float2(0.f, 0.f);
      if (idx < ib * I0) {
        const int r = I0 + idx % ib, c = idx / ib;
        for (int rp = I0; rp <= r; ++rp) {
          const float2 p = c_mul(XL(r, rp), XU(rp, c));
          xv[q].x -= p.x;
          xv[q].y -= p.y;
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < (CB * MAXN + C32_THREADS - 1) / C32_THREADS; ++q) {
      const int idx = t + q * C32_THREADS;
      if (idx < ib * I0) XU(I0 + idx % ib, idx / ib) = xv[q];
    }
    __syncthreads();
  }
  const float sgn = conj_out ? -1.f : 1.f;
  for (int e = t; e < n * n; e += C32_THREADS) {
    const int r = e / n, c = e - (e / n) * n;
    const float2 x = c <= r ? XL(r, c) : make_float2(0.f, 0.f);
    Out[e] = make_double2((double)x.x, (double)(sgn * x.y));
    if (Out32) Out32[e] = make_float2(x.x, sgn * x.y);
  }
#undef UL
#undef XU
#undef XL
}

// Triangular products on 8 x 8 output tiles (64 threads, one output each), K staged through
// shared memory in chunks of 32 with coalesced loads:
//   MODE 0: C = S M^H             C_ij = sum_{k <= j} S_ik conj(M_jk)          (all tiles, FP64)
//   MODE 1: C = M T (lower part)  C_ij = sum_{k <= i} M_ik T_kj, i >= j          (FP64)
//   MODE 2: C = conj(B - Phi(A - I) B) with A = S2 (lower) and B = M1:
//           C_ij = conj(B_ij - sum_{j <= k <= i} Phi_ik B_kj), Phi_ik = A_ik for k < i and
//           (A_ii - 1)/2 for k = i; i >= j, 0 above; C = I once *status is set.  Phi is
//           O(eps_32 kappa), so FP32 products keep the 24-bit accuracy of the rotation.
// MODE 2 also writes an FP32 copy of C to C32 when it is given.
template <int MODE>
__global__ void __launch_bounds__(64) k_tri_product(const double2* __restrict__ A, const double2* __restrict__ B,
                                                    int n, const int* __restrict__ status, double2* __restrict__ C,
                                                    float2* __restrict__ C32) {
  constexpr int KC = 32;
  __shared__ double2 As[8][KC + 1];
  __shared__ double2 Bs[8][KC + 1];                                  // Bs[j][k]
  const int ty = threadIdx.x >> 3, tx = threadIdx.x & 7;
  const int I = blockIdx.y * 8, J = blockIdx.x * 8;
  const int i = I + ty, j = J + tx;
  if (MODE == 2 && *status != 0) {
    if (i < n && j < n) {
      C[(size_t)i * n + j] = make_double2(i == j ? 1.0 : 0.0, 0.0);
      if (C32) C32[(size_t)i * n + j] = make_float2(i == j ? 1.f : 0.f, 0.f);
    }
    return;
  }
  if (MODE != 0 && J > I) {                                          // strictly upper tile
    if (MODE == 2 && i < n && j < n) {
      C[(size_t)i * n + j] = make_double2(0.0, 0.0);
      if (C32) C32[(size_t)i * n + j] = make_float2(0.f, 0.f);
    }
    return;
  }
  // k range of the tile
  const int k0 = MODE == 2 ? J : 0;
  const int k1 = min(n, MODE == 0 ? J + 8 : I + 8);
  using R = typename std::conditional<MODE == 2, float, double>::type;
  R re = 0, im = 0;
  for (int kc = k0; kc < k1; kc += KC) {
    for (int e = threadIdx.x; e < 8 * KC; e += 64) {
      const int r = e / KC, k = kc + e % KC;
      As[r][e % KC] = (I + r < n && k < k1) ? A[(size_t)(I + r) * n + k] : make_double2(0.0, 0.0);
      if (MODE == 0) {
        Bs[r][e % KC] = (J + r < n && k < k1) ? B[(size_t)(J + r) * n + k] : make_double2(0.0, 0.0);
      } else {
        const int kk = kc + e / 8, jj = e % 8;                        // B rows k, columns J..J+7
        Bs[jj][e / 8] = (kk < k1 && J + jj < n) ? B[(size_t)kk * n + J + jj] : make_double2(0.0, 0.0);
      }
    }
    __syncthreads();
    const int kend = min(KC, k1 - kc);
    for (int kk = 0; kk < kend; ++kk) {
      const int k = kc + kk;
      const double2 a = As[ty][kk], b = Bs[tx][kk];
      if (MODE == 0) {
        if (k <= j) {
          re += a.x * b.x + a.y * b.y;
          im += a.y * b.x - a.x * b.y;
        }
      } else if (MODE == 1) {
        if (k <= i) {
          re += a.x * b.x - a.y * b.y;
          im += a.x * b.y + a.y * b.x;
        }
      } else {
        if (k >= j && k <= i) {
          R ax = (R)a.x, ay = (R)a.y;
          if (k == i) {                                              // Phi_ii = (A_ii - 1) / 2
            ax = (R)(0.5 * (a.x - 1.0));
            ay = 0;
          }
          const R bx = (R)b.x, by = (R)b.y;
          re += ax * bx - ay * by;
          im += ax * by + ay * bx;
        }
      }
    }
    __syncthreads();
  }
  if (i >= n || j >= n) return;
  if (MODE == 0) {
    C[(size_t)i * n + j] = make_double2((double)re, (double)im);
  } else if (MODE == 1) {
    if (j <= i) C[(size_t)i * n + j] = make_double2((double)re, (double)im);
  } else {
    double2 c = make_double2(0.0, 0.0);
    if (j <= i) {
      const double2 bij = B[(size_t)i * n + j];
      c = make_double2(bij.x - (double)re, -(bij.y - (double)im));
    }
    C[(size_t)i * n + j] = c;
    if (C32) C32[(size_t)i * n + j] = make_float2((float)c.x, (float)c.y);
  }
}

}  // namespace

// M1, T, S2 (n^2 complex128 each), then for n > C32_MAXN the FP32 square array in global memory
size_t cholesky_mixed_workspace(int n) {
  return (size_t)3 * n * n + (n > C32_MAXN ? ((size_t)n * (n + 1) + 1) / 2 : 0);
}

void cholesky_inverse_mixed(const double2* S, double2* M, int n, double tol, double2* work, int* status,
                            cudaStream_t s, float2* M32, bool refine) {
  if (n > C32_MAXN_GLOBAL) fail(KS_ERR_ARG, "cholesky_inverse_mixed: n=%d > %d", n, C32_MAXN_GLOBAL);
  const bool glb = n > C32_MAXN;
  const size_t smem = glb ? 0 : (size_t)n * (n + 1) * sizeof(float2);   // square [n][n+1]
  static bool attr_set = false;
  if (!attr_set) {
    KS_CUDA(cudaFuncSetAttribute(k_chol32_inverse<C32_MAXN, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)((size_t)C32_MAXN * (C32_MAXN + 1) * sizeof(float2))));
    attr_set = true;
  }
  double2* M1 = work;
  double2* T = work + (size_t)n * n;
  double2* S2 = work + (size_t)2 * n * n;
  float2* gU = reinterpret_cast<float2*>(work + (size_t)3 * n * n);
  auto factor = [&](int conj_out, double2* out, float2* out32) {
    if (glb)
      k_chol32_inverse<C32_MAXN_GLOBAL, true><<<1, C32_THREADS, 0, s>>>(S, n, tol, conj_out, status, out, out32, gU);
    else
      k_chol32_inverse<C32_MAXN, false><<<1, C32_THREADS, smem, s>>>(S, n, tol, conj_out, status, out, out32, nullptr);
    KS_CHECK_LAUNCH();
  };
  if (!refine) {                                                     // the FP32 factor itself
    factor(1, M, M32);
    return;
  }
  const int nt = (n + 7) / 8;
  const dim3 grid(nt, nt);
  factor(0, M1, nullptr);
  k_tri_product<0><<<grid, 64, 0, s>>>(S, M1, n, status, T, nullptr);
  KS_CHECK_LAUNCH();
  k_tri_product<1><<<grid, 64, 0, s>>>(M1, T, n, status, S2, nullptr);   // S2 = M1 S M1^H (lower)
  KS_CHECK_LAUNCH();
  k_tri_product<2><<<grid, 64, 0, s>>>(S2, M1, n, status, M, M32);
  KS_CHECK_LAUNCH();
}

}  // namespace ks
