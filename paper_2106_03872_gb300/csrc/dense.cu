// Dense linear algebra of the state-space rotations (Sec. "Ground-state solution":
// orthogonalisation and subspace diagonalisation): overlap GEMMs, rotations, FP64
// Cholesky + triangular inverse, a cyclic Jacobi Hermitian eigensolver (FP64 path), and the
// FP64 Rayleigh quotients / sorting that finish the mixed path's FP32 eigenvectors.
// CUDA-core versions templated on the real type of the states.
#include <algorithm>
#include <type_traits>

#include "kernels.h"

namespace ks {

namespace {

constexpr int GT = 32;   // output tile
constexpr int KT = 16;   // K step

// part[ks][i][j] = sum_{k in chunk ks} conj(A[i][k]) B[j][k]
template <typename T>
__global__ void __launch_bounds__(256) k_gemm_cn(const cplx<T>* __restrict__ A, int lda, const cplx<T>* __restrict__ B,
                                                 int ldb, int m, int n, int K, int kchunk, double2* __restrict__ part) {
  using C = cplx<T>;
  __shared__ C As[GT][KT + 1];
  __shared__ C Bs[GT][KT + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int i0 = blockIdx.y * GT, j0 = blockIdx.x * GT;
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(K, kbeg + kchunk);
  T acc[2][2][2] = {};
  for (int k0 = kbeg; k0 < kend; k0 += KT) {
    for (int e = threadIdx.x; e < GT * KT; e += 256) {
      const int r = e / KT, kk = e % KT;
      const int k = k0 + kk;
      As[r][kk] = (i0 + r < m && k < kend) ? A[(size_t)(i0 + r) * lda + k] : mk<C>(T(0), T(0));
      Bs[r][kk] = (j0 + r < n && k < kend) ? B[(size_t)(j0 + r) * ldb + k] : mk<C>(T(0), T(0));
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < KT; ++kk) {
      C a[2], b[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        a[u] = As[ty + 16 * u][kk];
        b[u] = Bs[tx + 16 * u][kk];
      }
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 2; ++v) {
          acc[u][v][0] += a[u].x * b[v].x + a[u].y * b[v].y;
          acc[u][v][1] += a[u].x * b[v].y - a[u].y * b[v].x;
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const int i = i0 + ty + 16 * u, j = j0 + tx + 16 * v;
      if (i < m && j < n)
        part[((size_t)blockIdx.z * m + i) * n + j] = make_double2((double)acc[u][v][0], (double)acc[u][v][1]);
    }
}

__global__ void k_reduce_parts(const double2* __restrict__ part, int nks, size_t mn, double2* __restrict__ out) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < mn; e += (size_t)gridDim.x * blockDim.x) {
    double2 s = make_double2(0.0, 0.0);
    for (int k = 0; k < nks; ++k) {
      const double2 p = part[(size_t)k * mn + e];
      s.x += p.x;
      s.y += p.y;
    }
    out[e] = s;
  }
}

// Y[i][k] = sum_j M[i][j] X[j][k]; tile 32 rows x 64 columns, each thread 2 x 4 outputs.
template <typename T>
__global__ void __launch_bounds__(256) k_rotate(const double2* __restrict__ M, int nin, const cplx<T>* __restrict__ X,
                                                const cplx<T>* __restrict__ X2, int nin1, int ldx, cplx<T>* __restrict__ Y,
                                                int ldy, int m, int K) {
  using C = cplx<T>;
  __shared__ C Ms[32][KT + 1];
  __shared__ C Xs[KT][64 + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int i0 = blockIdx.y * 32, k0 = blockIdx.x * 64;
  T acc[2][4][2] = {};
  for (int j0 = 0; j0 < nin; j0 += KT) {
    for (int e = threadIdx.x; e < 32 * KT; e += 256) {
      const int r = e / KT, jj = e % KT;
      const double2 v = (i0 + r < m && j0 + jj < nin) ? M[(size_t)(i0 + r) * nin + j0 + jj] : make_double2(0.0, 0.0);
      Ms[r][jj] = mk<C>(T(v.x), T(v.y));
    }
    for (int e = threadIdx.x; e < KT * 64; e += 256) {
      const int jj = e / 64, c = e % 64;
      const int j = j0 + jj;
      Xs[jj][c] = (j < nin && k0 + c < K)
                      ? (j < nin1 ? X[(size_t)j * ldx + k0 + c] : X2[(size_t)(j - nin1) * ldx + k0 + c])
                      : mk<C>(T(0), T(0));
    }
    __syncthreads();
#pragma unroll
    for (int jj = 0; jj < KT; ++jj) {
      C a[2], x[4];
#pragma unroll
      for (int u = 0; u < 2; ++u) a[u] = Ms[ty + 16 * u][jj];
#pragma unroll
      for (int v = 0; v < 4; ++v) x[v] = Xs[jj][tx + 16 * v];
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          acc[u][v][0] += a[u].x * x[v].x - a[u].y * x[v].y;
          acc[u][v][1] += a[u].x * x[v].y + a[u].y * x[v].x;
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int i = i0 + ty + 16 * u, k = k0 + tx + 16 * v;
      if (i < m && k < K) Y[(size_t)i * ldy + k] = mk<C>(acc[u][v][0], acc[u][v][1]);
    }
}

__global__ void k_hermitize(double2* A, int n) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += gridDim.x * blockDim.x) {
    const int i = e / n, j = e % n;
    if (i < j) {
      const double2 a = A[i * n + j], b = A[j * n + i];
      const double2 h = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
      A[i * n + j] = h;
      A[j * n + i] = make_double2(h.x, -h.y);
    } else if (i == j) {
      A[i * n + i].y = 0.0;
    }
  }
}

__device__ __forceinline__ double2 zmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ double2 zconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 zscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 zadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 zsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

// Left-looking Cholesky of the lower triangle of A (in place), then M = conj(L^{-1}).
// A diagonal pivot d_j <= tol * S_jj (the squared norm of state j left after removing
// the earlier states) marks S as not positive definite: status = j + 1, M = I.
__global__ void __launch_bounds__(512) k_cholesky_inverse(double2* __restrict__ A, double2* __restrict__ M, int n,
                                                          double tol, int* __restrict__ status) {
  __shared__ int bad;
  __shared__ double ljj;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    for (int i = j + threadIdx.x; i < n; i += blockDim.x) {
      double2 t = A[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) t = zsub(t, zmul(A[(size_t)i * n + k], zconj(A[(size_t)j * n + k])));
      if (i == j) {
        const double sjj = A[(size_t)j * n + j].x;
        if (!(t.x > tol * sjj) || !isfinite(t.x)) bad = j + 1;
      }
      A[(size_t)i * n + j] = t;
    }
    __syncthreads();
    if (bad) break;
    if (threadIdx.x == 0) {
      ljj = sqrt(A[(size_t)j * n + j].x);
      A[(size_t)j * n + j] = make_double2(ljj, 0.0);
    }
    __syncthreads();
    const double inv = 1.0 / ljj;
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) A[(size_t)i * n + j] = zscale(A[(size_t)i * n + j], inv);
    __syncthreads();
  }
  if (bad) {
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) M[e] = make_double2((e / n == e % n) ? 1.0 : 0.0, 0.0);
    if (threadIdx.x == 0) *status = bad;
    return;
  }
  // X = L^{-1}, one column per thread: x_i = (delta_ic - sum_{k=c}^{i-1} L_ik x_k) / L_ii
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    for (int i = c; i < n; ++i) {
      double2 t = make_double2(i == c ? 1.0 : 0.0, 0.0);
      for (int k = c; k < i; ++k) t = zsub(t, zmul(A[(size_t)i * n + k], M[(size_t)k * n + c]));
      M[(size_t)i * n + c] = zscale(t, 1.0 / A[(size_t)i * n + i].x);
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, c = e % n;
    M[e] = (i < c) ? make_double2(0.0, 0.0) : zconj(M[e]);
  }
}

// Cyclic Jacobi for a Hermitian n x n matrix (n <= 512) in one CTA, parallel
// round-robin ordering (n/2 disjoint rotations per round).  Rotation of the (p, q) pair:
// with a_pq = |b| e^{i phi}, J = [[c, s e^{i phi}], [-s e^{-i phi}, c]] where (c, s) is the
// real symmetric Schur rotation of [[a_pp, |b|], [|b|, a_qq]]; A <- J^H A J, V <- V J.
__global__ void __launch_bounds__(1024) k_jacobi(double2* __restrict__ A, double2* __restrict__ V,
                                                 double* __restrict__ eig, double2* __restrict__ Vt, int n) {
  __shared__ int sp[256], sq[256];
  __shared__ double sc[256], ss[256];
  __shared__ double2 se[256];
  __shared__ int srot;
  __shared__ double sthr;
  __shared__ double red[32];
  const int P = n + (n & 1);
  const int np = P / 2;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) V[e] = make_double2((e / n == e % n) ? 1.0 : 0.0, 0.0);
  // threshold from the Frobenius norm
  double f = 0.0;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) f += A[e].x * A[e].x + A[e].y * A[e].y;
  for (int o = 16; o > 0; o >>= 1) f += __shfl_down_sync(0xffffffffu, f, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = f;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0;
    for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) s += red[w];
    sthr = 1e-15 * sqrt(s);
  }
  __syncthreads();
  for (int sweep = 0; sweep < 60; ++sweep) {
    if (threadIdx.x == 0) srot = 0;
    __syncthreads();
    for (int r = 0; r < P - 1; ++r) {
      if (threadIdx.x < np) {
        const int k = threadIdx.x;
        const int pa = k, pb = P - 1 - k;
        const int ua = (pa == 0) ? 0 : 1 + ((pa - 1 + r) % (P - 1));
        const int ub = (pb == 0) ? 0 : 1 + ((pb - 1 + r) % (P - 1));
        const int p = min(ua, ub), q = max(ua, ub);
        int active = 0;
        if (q < n) {
          const double2 b = A[(size_t)p * n + q];
          const double mag = hypot(b.x, b.y);
          if (mag > sthr) {
            const double alpha = A[(size_t)p * n + p].x, gamma = A[(size_t)q * n + q].x;
            const double tau = (gamma - alpha) / (2.0 * mag);
            const double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            const double c = 1.0 / sqrt(1.0 + t * t);
            sc[k] = c;
            ss[k] = t * c;
            se[k] = make_double2(b.x / mag, b.y / mag);
            active = 1;
            srot = 1;
          }
        }
        sp[k] = p;
        sq[k] = active ? q : -1;
      }
      __syncthreads();
      // rows: A <- J^H A
      for (int job = threadIdx.x; job < np * n; job += blockDim.x) {
        const int k = job / n, j = job % n;
        const int q = sq[k];
        if (q < 0) continue;
        const int p = sp[k];
        const double c = sc[k], s = ss[k];
        const double2 e = se[k];
        const double2 ap = A[(size_t)p * n + j], aq = A[(size_t)q * n + j];
        A[(size_t)p * n + j] = zsub(zscale(ap, c), zscale(zmul(e, aq), s));
        A[(size_t)q * n + j] = zadd(zscale(zmul(zconj(e), ap), s), zscale(aq, c));
      }
      __syncthreads();
      // columns: A <- A J, V <- V J
      for (int job = threadIdx.x; job < np * n; job += blockDim.x) {
        const int k = job / n, i = job % n;
        const int q = sq[k];
        if (q < 0) continue;
        const int p = sp[k];
        const double c = sc[k], s = ss[k];
        const double2 e = se[k];
        double2 ap = A[(size_t)i * n + p], aq = A[(size_t)i * n + q];
        A[(size_t)i * n + p] = zsub(zscale(ap, c), zscale(zmul(zconj(e), aq), s));
        A[(size_t)i * n + q] = zadd(zscale(zmul(e, ap), s), zscale(aq, c));
        ap = V[(size_t)i * n + p];
        aq = V[(size_t)i * n + q];
        V[(size_t)i * n + p] = zsub(zscale(ap, c), zscale(zmul(zconj(e), aq), s));
        V[(size_t)i * n + q] = zadd(zscale(zmul(e, ap), s), zscale(aq, c));
      }
      __syncthreads();
    }
    if (srot == 0) break;
    __syncthreads();
  }
  // sort ascending (ties by index), phase-fix each eigenvector, write rows of Vt
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double ei = A[(size_t)i * n + i].x;
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const double ej = A[(size_t)j * n + j].x;
      rank += (ej < ei) || (ej == ei && j < i);
    }
    int kmax = 0;
    double best = -1.0;
    for (int j = 0; j < n; ++j) {
      const double2 v = V[(size_t)j * n + i];
      const double m2 = v.x * v.x + v.y * v.y;
      if (m2 > best) {
        best = m2;
        kmax = j;
      }
    }
    const double2 vk = V[(size_t)kmax * n + i];
    const double mag = sqrt(best);
    const double2 ph = make_double2(vk.x / mag, -vk.y / mag);
    eig[rank] = ei;
    for (int j = 0; j < n; ++j) Vt[(size_t)rank * n + j] = zmul(V[(size_t)j * n + i], ph);
  }
}

// The same parallel round-robin Jacobi in FP32 for the mixed path's subspace problems of
// 128 < n <= 256 (the one-CTA Householder solver holds n <= 128 in shared memory): A (FP32,
// destroyed) and the eigenvector columns V in global memory, L2-resident; rotations of pairs
// whose coupling is below 1e-6 |A|_F are skipped (FP32 rounding of a rotated entry is ~6e-8
// |A|), so the sweeps stop once the off-diagonal part is at FP32 level.  No sorting: the caller
// takes FP64 Rayleigh quotients of the vectors, then sorts (eigh_jacobi_mixed).
__device__ __forceinline__ float2 cmulf(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ float2 cconjf(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscalef(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

__global__ void __launch_bounds__(1024) k_jacobi32(float2* __restrict__ A, float2* __restrict__ V, int n) {
  __shared__ int sp[256], sq[256];
  __shared__ float sc[256], ss[256];
  __shared__ float2 se[256];
  __shared__ int srot;
  __shared__ float sthr;
  __shared__ float red[32];
  const int P = n + (n & 1);
  const int np = P / 2;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) V[e] = make_float2((e / n == e % n) ? 1.f : 0.f, 0.f);
  float f = 0.f;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) f += A[e].x * A[e].x + A[e].y * A[e].y;
  for (int o = 16; o > 0; o >>= 1) f += __shfl_down_sync(0xffffffffu, f, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = f;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) t += red[w];
    sthr = 1e-6f * sqrtf(t);
  }
  __syncthreads();
  for (int sweep = 0; sweep < 40; ++sweep) {
    if (threadIdx.x == 0) srot = 0;
    __syncthreads();
    for (int r = 0; r < P - 1; ++r) {
      if (threadIdx.x < np) {
        const int k = threadIdx.x;
        const int pa = k, pb = P - 1 - k;
        const int ua = (pa == 0) ? 0 : 1 + ((pa - 1 + r) % (P - 1));
        const int ub = (pb == 0) ? 0 : 1 + ((pb - 1 + r) % (P - 1));
        const int p = min(ua, ub), q = max(ua, ub);
        int active = 0;
        if (q < n) {
          const float2 b = A[(size_t)p * n + q];
          const float mag = hypotf(b.x, b.y);
          if (mag > sthr) {
            const float alpha = A[(size_t)p * n + p].x, gamma = A[(size_t)q * n + q].x;
            const float tau = (gamma - alpha) / (2.f * mag);
            const float t = (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(1.f + tau * tau));
            const float c = 1.f / sqrtf(1.f + t * t);
            sc[k] = c;
            ss[k] = t * c;
            se[k] = make_float2(b.x / mag, b.y / mag);
            active = 1;
            srot = 1;
          }
        }
        sp[k] = p;
        sq[k] = active ? q : -1;
      }
      __syncthreads();
      for (int job = threadIdx.x; job < np * n; job += blockDim.x) {     // rows: A <- J^H A
        const int k = job / n, j = job % n;
        const int q = sq[k];
        if (q < 0) continue;
        const int p = sp[k];
        const float c = sc[k], sv = ss[k];
        const float2 e = se[k];
        const float2 ap = A[(size_t)p * n + j], aq = A[(size_t)q * n + j];
        A[(size_t)p * n + j] = cscalef(ap, c) - cscalef(cmulf(e, aq), sv);
        A[(size_t)q * n + j] = cscalef(cmulf(cconjf(e), ap), sv) + cscalef(aq, c);
      }
      __syncthreads();
      for (int job = threadIdx.x; job < np * n; job += blockDim.x) {     // columns: A <- A J, V <- V J
        const int k = job / n, i = job % n;
        const int q = sq[k];
        if (q < 0) continue;
        const int p = sp[k];
        const float c = sc[k], sv = ss[k];
        const float2 e = se[k];
        float2 ap = A[(size_t)i * n + p], aq = A[(size_t)i * n + q];
        A[(size_t)i * n + p] = cscalef(ap, c) - cscalef(cmulf(cconjf(e), aq), sv);
        A[(size_t)i * n + q] = cscalef(cmulf(e, ap), sv) + cscalef(aq, c);
        ap = V[(size_t)i * n + p];
        aq = V[(size_t)i * n + q];
        V[(size_t)i * n + p] = cscalef(ap, c) - cscalef(cmulf(cconjf(e), aq), sv);
        V[(size_t)i * n + q] = cscalef(cmulf(e, ap), sv) + cscalef(aq, c);
      }
      __syncthreads();
    }
    if (srot == 0) break;
    __syncthreads();
  }
}

__global__ void k_c128_to_c64(const double2* __restrict__ in, float2* __restrict__ out, size_t n) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    out[e] = make_float2((float)in[e].x, (float)in[e].y);
}
__global__ void k_c64_to_c128(const float2* __restrict__ in, double2* __restrict__ out, size_t n) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    out[e] = make_double2((double)in[e].x, (double)in[e].y);
}

// lam[i] = v_i^H H v_i / v_i^H v_i in FP64 (column i of V), one CTA per i.
__global__ void k_rayleigh_quotients(const double2* __restrict__ H, const double2* __restrict__ V, int n,
                                     double* __restrict__ lam) {
  const int i = blockIdx.x;
  __shared__ double2 vi[512];
  __shared__ double red[2][32];
  for (int k = threadIdx.x; k < n; k += blockDim.x) vi[k] = V[(size_t)k * n + i];
  __syncthreads();
  double num = 0.0, den = 0.0;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int j = e / n, k = e % n;
    // conj(v_j) H_jk v_k
    const double2 hv = zmul(H[e], vi[k]);
    num += vi[j].x * hv.x + vi[j].y * hv.y;
    if (j == k) den += vi[k].x * vi[k].x + vi[k].y * vi[k].y;
  }
  for (int o = 16; o > 0; o >>= 1) {
    num += __shfl_down_sync(0xffffffffu, num, o);
    den += __shfl_down_sync(0xffffffffu, den, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = num;
    red[1][threadIdx.x >> 5] = den;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a += red[0][w];
      b += red[1][w];
    }
    lam[i] = a / b;
  }
}

// C = opA(A) opB(B) for n x n complex128 matrices (row-major).  flags: bit 0 conjugates A,
// bit 1 transposes B (opB(B)_kj = B_jk), bit 2 conjugates B.  8 x 8 output tiles, K staged
// through shared memory 32 at a time.  MIXED: products and sums in FP32 inside a 32-wide K
// chunk, FP64 across chunks; otherwise FP64 throughout.
template <bool MIXED>
__global__ void __launch_bounds__(64) k_small_product(const double2* __restrict__ A, const double2* __restrict__ B,
                                                      int n, int flags, double2* __restrict__ C) {
  constexpr int KC = 32;
  using R = typename std::conditional<MIXED, float, double>::type;
  __shared__ double2 As[8][KC + 1];
  __shared__ double2 Bs[8][KC + 1];                                  // Bs[j][k] = opB(B)_kj
  const int ty = threadIdx.x >> 3, tx = threadIdx.x & 7;
  const int I = blockIdx.y * 8, J = blockIdx.x * 8;
  const bool ca = flags & 1, tb = flags & 2, cb = flags & 4;
  double re = 0.0, im = 0.0;
  for (int kc = 0; kc < n; kc += KC) {
    for (int e = threadIdx.x; e < 8 * KC; e += 64) {
      const int r = e / KC, k = kc + e % KC;
      double2 a = (I + r < n && k < n) ? A[(size_t)(I + r) * n + k] : make_double2(0.0, 0.0);
      if (ca) a.y = -a.y;
      As[r][e % KC] = a;
      double2 b;
      int jj, kk;
      if (tb) {                                                      // opB(B)_kj = B_jk: rows J..J+7
        jj = r;
        kk = e % KC;
        b = (J + r < n && k < n) ? B[(size_t)(J + r) * n + k] : make_double2(0.0, 0.0);
      } else {                                                       // B rows k, columns J..J+7
        jj = e % 8;
        kk = e / 8;
        b = (kc + kk < n && J + jj < n) ? B[(size_t)(kc + kk) * n + J + jj] : make_double2(0.0, 0.0);
      }
      if (cb) b.y = -b.y;
      Bs[jj][kk] = b;
    }
    __syncthreads();
    R cr = 0, ci = 0;
#pragma unroll 8
    for (int kk = 0; kk < KC; ++kk) {
      const double2 a = As[ty][kk], b = Bs[tx][kk];
      const R ax = (R)a.x, ay = (R)a.y, bx = (R)b.x, by = (R)b.y;
      cr += ax * bx - ay * by;
      ci += ax * by + ay * bx;
    }
    re += (double)cr;
    im += (double)ci;
    __syncthreads();
  }
  const int i = I + ty, j = J + tx;
  if (i < n && j < n) C[(size_t)i * n + j] = make_double2(re, im);
}

// Mcat = [ (I + alpha Lambda) C | -alpha C ] (n x 2n): one steepest-descent step of the Ritz
// block, psi_new = Mcat [psi; H psi] with the Ritz rotation C folded in.
__global__ void k_sd_matrix(const double2* __restrict__ C, const double* __restrict__ eig, double alpha, int n,
                            double2* __restrict__ Mcat) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += gridDim.x * blockDim.x) {
    const int i = e / n, j = e - (e / n) * n;
    const double2 c = C[e];
    const double f = 1.0 + alpha * eig[i];
    Mcat[(size_t)i * 2 * n + j] = make_double2(f * c.x, f * c.y);
    Mcat[(size_t)i * 2 * n + n + j] = make_double2(-alpha * c.x, -alpha * c.y);
  }
}

// Sort by lam (ties by index), normalise, fix phases; Vt row r = eigenvector of rank r.
__global__ void k_sort_vectors(const double* __restrict__ lam, const double2* __restrict__ V, int n,
                               double* __restrict__ eig, double2* __restrict__ Vt) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double li = lam[i];
    int rank = 0;
    for (int j = 0; j < n; ++j) rank += (lam[j] < li) || (lam[j] == li && j < i);
    int kmax = 0;
    double best = -1.0, nrm = 0.0;
    for (int j = 0; j < n; ++j) {
      const double2 v = V[(size_t)j * n + i];
      const double m2 = v.x * v.x + v.y * v.y;
      nrm += m2;
      if (m2 > best) {
        best = m2;
        kmax = j;
      }
    }
    const double2 vk = V[(size_t)kmax * n + i];
    const double mag = sqrt(best);
    const double sc = 1.0 / (mag * sqrt(nrm));
    const double2 ph = make_double2(vk.x * sc, -vk.y * sc);
    eig[rank] = li;
    for (int j = 0; j < n; ++j) Vt[(size_t)rank * n + j] = zmul(V[(size_t)j * n + i], ph);
  }
}

}  // namespace

template <typename T>
void gemm_cn(const cplx<T>* A, int lda, const cplx<T>* B, int ldb, int m, int n, int K, double2* part,
             size_t part_elems, double2* out, cudaStream_t s) {
  const int tm = (m + GT - 1) / GT, tn = (n + GT - 1) / GT;
  int ks = std::max(1, 304 / (tm * tn));
  ks = std::min(ks, std::max(1, K / 256));
  ks = std::min<long>(ks, (long)(part_elems / ((size_t)m * n)));
  if (ks < 1) fail(KS_ERR_ARG, "gemm_cn: partial buffer too small");
  int kchunk = (K + ks - 1) / ks;
  kchunk = (kchunk + KT - 1) / KT * KT;
  ks = (K + kchunk - 1) / kchunk;
  dim3 g(tn, tm, ks);
  k_gemm_cn<T><<<g, 256, 0, s>>>(A, lda, B, ldb, m, n, K, kchunk, part);
  KS_CHECK_LAUNCH();
  const size_t mn = (size_t)m * n;
  k_reduce_parts<<<(unsigned)std::min<size_t>((mn + 255) / 256, 1024), 256, 0, s>>>(part, ks, mn, out);
  KS_CHECK_LAUNCH();
}

template <typename T>
void rotate(const double2* M, int nin, const cplx<T>* X, const cplx<T>* X2, int nin1, int ldx, cplx<T>* Y, int ldy,
            int m, int K, cudaStream_t s) {
  if (!X2) nin1 = nin;
  dim3 g((K + 63) / 64, (m + 31) / 32);
  k_rotate<T><<<g, 256, 0, s>>>(M, nin, X, X2, nin1, ldx, Y, ldy, m, K);
  KS_CHECK_LAUNCH();
}

void hermitize(double2* A, int n, cudaStream_t s) {
  k_hermitize<<<std::max(1, std::min(1024, (n * n + 255) / 256)), 256, 0, s>>>(A, n);
  KS_CHECK_LAUNCH();
}

void cholesky_inverse(double2* A, double2* M, int n, int* status, cudaStream_t s) {
  // tolerance on the relative pivot: FP64 states give S to ~1e-16, FP32 states to ~1e-7.
  cholesky_inverse_tol(A, M, n, 1e-12, status, s);
}

void cholesky_inverse_tol(double2* A, double2* M, int n, double tol, int* status, cudaStream_t s) {
  if (n > 512) fail(KS_ERR_ARG, "cholesky: n=%d > 512", n);
  k_cholesky_inverse<<<1, 512, 0, s>>>(A, M, n, tol, status);
  KS_CHECK_LAUNCH();
}

void eigh_jacobi_mixed(const double2* A, double2* V, double* lam, double* eig, double2* Vt, float2* work, int n,
                       cudaStream_t s) {
  if (n > 256 || n < 1) fail(KS_ERR_ARG, "eigh_jacobi_mixed: n=%d not in [1, 256]", n);
  const size_t nn = (size_t)n * n;
  float2* A32 = work;
  float2* V32 = work + nn;
  const unsigned nb = (unsigned)std::min<size_t>((nn + 255) / 256, 1024);
  k_c128_to_c64<<<nb, 256, 0, s>>>(A, A32, nn);
  KS_CHECK_LAUNCH();
  k_jacobi32<<<1, 1024, 0, s>>>(A32, V32, n);
  KS_CHECK_LAUNCH();
  k_c64_to_c128<<<nb, 256, 0, s>>>(V32, V, nn);
  KS_CHECK_LAUNCH();
  k_rayleigh_quotients<<<n, 256, 0, s>>>(A, V, n, lam);
  KS_CHECK_LAUNCH();
  k_sort_vectors<<<1, 128, 0, s>>>(lam, V, n, eig, Vt);
  KS_CHECK_LAUNCH();
}

void eigh_mixed(const double2* A, double2* V, double* lam, double* eig, double2* Vt, int n, cudaStream_t s) {
  eigh_householder_f32(A, V, n, s);
  k_rayleigh_quotients<<<n, 256, 0, s>>>(A, V, n, lam);
  KS_CHECK_LAUNCH();
  k_sort_vectors<<<1, 128, 0, s>>>(lam, V, n, eig, Vt);
  KS_CHECK_LAUNCH();
}

void small_product(const double2* A, const double2* B, int n, int flags, bool mixed, double2* C, cudaStream_t s) {
  const dim3 grid((n + 7) / 8, (n + 7) / 8);
  if (mixed)
    k_small_product<true><<<grid, 64, 0, s>>>(A, B, n, flags, C);
  else
    k_small_product<false><<<grid, 64, 0, s>>>(A, B, n, flags, C);
  KS_CHECK_LAUNCH();
}

void sd_matrix(const double2* C, const double* eig, double alpha, int n, double2* Mcat, cudaStream_t s) {
  k_sd_matrix<<<std::max(1, std::min(256, (n * n + 255) / 256)), 256, 0, s>>>(C, eig, alpha, n, Mcat);
  KS_CHECK_LAUNCH();
}

void jacobi_eigh(double2* A, double2* V, double* eig, double2* Vt, int n, cudaStream_t s) {
  if (n > 512) fail(KS_ERR_ARG, "jacobi: n=%d > 512", n);
  k_jacobi<<<1, 1024, 0, s>>>(A, V, eig, Vt, n);
  KS_CHECK_LAUNCH();
}

template void gemm_cn<float>(const float2*, int, const float2*, int, int, int, int, double2*, size_t, double2*,
                             cudaStream_t);
template void gemm_cn<double>(const double2*, int, const double2*, int, int, int, int, double2*, size_t, double2*,
                              cudaStream_t);
template void rotate<float>(const double2*, int, const float2*, const float2*, int, int, float2*, int, int, int,
                            cudaStream_t);
template void rotate<double>(const double2*, int, const double2*, const double2*, int, int, double2*, int, int, int,
                             cudaStream_t);

}  // namespace ks
