// Hermitian eigen-decomposition of the Rayleigh-Ritz matrix on the mixed path (n <= 128),
// one CTA, FP32, matrix in shared memory:
//
//   1. Householder reduction A = Q T Q^H to a real symmetric tridiagonal T: for column k the
//      reflector H_k = I - tau_k v_k v_k^H (v_k[0] = 1) maps A[k+1:, k] to (beta_k, 0, ...)
//      with real beta_k; the trailing block is updated as A -= v w^H + w v^H with
//      w = tau A v - (tau/2)(w'^H v) v (the classic two-sided Hermitian update).
//   2. T is split where an off-diagonal element is negligible; every block's eigenvalues are
//      found by multisection on its Sturm count (8 lanes per eigenvalue, 9-way split per step).
//   3. Eigenvectors of each block by twisted factorization (forward and backward pivots,
//      twist index at the smallest |gamma|), then modified Gram-Schmidt inside clusters of
//      close eigenvalues of a block.
//   4. Back-transformation V = H_0 H_1 ... H_{n-2} Z.
//
// The FP32 vectors are written as complex128 columns; the caller takes the eigenvalues as
// FP64 Rayleigh quotients of these vectors on the FP64 matrix, then sorts and fixes phases.
#include "kernels.h"

namespace ks {

namespace {

constexpr int EH_MAXN = 128;
constexpr int EH_THREADS = 1024;

__device__ __forceinline__ float2 cm(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ float2 cmc(float2 a, float2 b) {   // conj(a) * b
  return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

// Number of eigenvalues of T[b0..b1] below x (Sturm count of the LDL^T pivots).
__device__ __forceinline__ int sturm_count(const float* d, const float* e2, int b0, int b1, float x, float pivmin) {
  int c = 0;
  float q = d[b0] - x;
  if (fabsf(q) < pivmin) q = -pivmin;
  c += q < 0.f;
  for (int i = b0 + 1; i <= b1; ++i) {
    q = d[i] - x - e2[i - 1] / q;
    if (fabsf(q) < pivmin) q = -pivmin;
    c += q < 0.f;
  }
  return c;
}

__global__ void __launch_bounds__(EH_THREADS, 1)
    k_eigh_householder(const double2* __restrict__ H, int n, double2* __restrict__ Vout) {
  extern __shared__ __align__(16) unsigned char esm[];
  const int ld = n + 1;
  float2* A = reinterpret_cast<float2*>(esm);                       // [n][ld], later Z
  float2* R = A + (size_t)EH_MAXN * (EH_MAXN + 1);                  // packed reflectors
  __shared__ float d[EH_MAXN], e[EH_MAXN], e2[EH_MAXN], lam[EH_MAXN];
  __shared__ float2 tau[EH_MAXN], wv[EH_MAXN];
  __shared__ int blk_lo[EH_MAXN], blk_hi[EH_MAXN];
  __shared__ float red[32][2];
  __shared__ float2 s_alpha, s_scale;
  __shared__ float s_beta;
  __shared__ int s_skip;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;

  for (int idx = t; idx < n * n; idx += EH_THREADS) {
    const int i = idx / n, j = idx - (idx / n) * n;
    const double2 h = H[idx];
    A[i * ld + j] = make_float2((float)h.x, i == j ? 0.f : (float)h.y);
  }
  __syncthreads();

  // ---- 1. tridiagonalization ---------------------------------------------------------------
  int roff = 0;
  for (int k = 0; k + 1 < n; ++k) {
    const int m = n - k - 1;                 // reflector length, rows k+1..n-1
    float2* v = R + roff;
    // xnorm^2 over x[1:], alpha = x[0]
    float s = 0.f;
    for (int i = 1 + t; i < m; i += EH_THREADS) {
      const float2 x = A[(k + 1 + i) * ld + k];
      s += x.x * x.x + x.y * x.y;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) red[warp][0] = s;
    __syncthreads();
    if (t == 0) {
      float xn2 = 0.f;
      for (int w = 0; w < EH_THREADS / 32; ++w) xn2 += red[w][0];
      const float2 al = A[(k + 1) * ld + k];
      d[k] = A[k * ld + k].x;
      if (xn2 == 0.f && al.y == 0.f) {
        tau[k] = make_float2(0.f, 0.f);
        e[k] = al.x;
        s_skip = 1;
      } else {
        const float beta = -copysignf(sqrtf(al.x * al.x + al.y * al.y + xn2), al.x);
        tau[k] = make_float2((beta - al.x) / beta, -al.y / beta);
        const float2 dn = make_float2(al.x - beta, al.y);          // 1 / (alpha - beta)
        const float inv = 1.f / (dn.x * dn.x + dn.y * dn.y);
        s_scale = make_float2(dn.x * inv, -dn.y * inv);
        e[k] = beta;
        s_skip = 0;
      }
    }
    __syncthreads();
    if (s_skip) {
      for (int i = t; i < m; i += EH_THREADS) v[i] = make_float2(i == 0 ? 1.f : 0.f, 0.f);
      roff += m;
      __syncthreads();
      continue;
    }
    const float2 sc = s_scale;
    for (int i = t; i < m; i += EH_THREADS) v[i] = (i == 0) ? make_float2(1.f, 0.f) : cm(A[(k + 1 + i) * ld + k], sc);
    __syncthreads();
    // w' = tau * A_t v  (A_t = A[k+1:, k+1:]); 8 threads per row
    const float2 tk = tau[k];
    {
      const int row = t >> 3, sub = t & 7;
      float2 acc = make_float2(0.f, 0.f);
      if (row < m) {
        const float2* arow = A + (k + 1 + row) * ld + (k + 1);
        for (int j = sub; j < m; j += 8) {
          const float2 a = arow[j], b = v[j];
          acc.x += a.x * b.x - a.y * b.y;
          acc.y += a.x * b.y + a.y * b.x;
        }
      }
      for (int o = 4; o > 0; o >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
      }
      if (row < m && sub == 0) wv[row] = cm(tk, acc);
    }
    __syncthreads();
    // alpha = -1/2 tau (w'^H v)
    {
      float2 p = make_float2(0.f, 0.f);
      for (int i = t; i < m; i += EH_THREADS) {
        const float2 q = cmc(wv[i], v[i]);
        p.x += q.x;
        p.y += q.y;
      }
      for (int o = 16; o > 0; o >>= 1) {
        p.x += __shfl_down_sync(0xffffffffu, p.x, o);
        p.y += __shfl_down_sync(0xffffffffu, p.y, o);
      }
      if (lane == 0) {
        red[warp][0] = p.x;
        red[warp][1] = p.y;
      }
      __syncthreads();
      if (t == 0) {
        float2 tot = make_float2(0.f, 0.f);
        for (int w = 0; w < EH_THREADS / 32; ++w) {
          tot.x += red[w][0];
          tot.y += red[w][1];
        }
        const float2 h = cm(tk, tot);
        s_alpha = make_float2(-0.5f * h.x, -0.5f * h.y);
      }
      __syncthreads();
    }
    {
      const float2 al = s_alpha;
      for (int i = t; i < m; i += EH_THREADS) {
        const float2 a = cm(al, v[i]);
        wv[i] = make_float2(wv[i].x + a.x, wv[i].y + a.y);
      }
    }
    __syncthreads();
    // A_t -= v w^H + w v^H
    for (int idx = t; idx < m * m; idx += EH_THREADS) {
      const int i = idx / m, j = idx - (idx / m) * m;
      const float2 vi = v[i], vj = v[j], wi = wv[i], wj = wv[j];
      float2 a = A[(k + 1 + i) * ld + (k + 1 + j)];
      // v_i conj(w_j) + w_i conj(v_j)
      a.x -= (vi.x * wj.x + vi.y * wj.y) + (wi.x * vj.x + wi.y * vj.y);
      a.y -= (vi.y * wj.x - vi.x * wj.y) + (wi.y * vj.x - wi.x * vj.y);
      if (i == j) a.y = 0.f;
      A[(k + 1 + i) * ld + (k + 1 + j)] = a;
    }
    roff += m;
    __syncthreads();
  }
  if (t == 0) {
    d[n - 1] = A[(n - 1) * ld + (n - 1)].x;
    e[n - 1] = 0.f;
  }
  __syncthreads();

  // ---- 2. split and eigenvalues ------------------------------------------------------------
  float tnorm = 0.f;
  if (t == 0) {
    // blocks: e[i] negligible against its neighbours -> boundary after i
    int b0 = 0;
    for (int i = 0; i < n; ++i) {
      const bool cut = (i == n - 1) || fabsf(e[i]) <= 1e-7f * (fabsf(d[i]) + fabsf(d[i + 1]) + 1e-30f);
      if (cut) {
        for (int j = b0; j <= i; ++j) {
          blk_lo[j] = b0;
          blk_hi[j] = i;
        }
        if (i < n - 1) e[i] = 0.f;
        b0 = i + 1;
      }
    }
    for (int i = 0; i < n; ++i) e2[i] = e[i] * e[i];
  }
  __syncthreads();
  for (int i = 0; i < n; ++i) tnorm = fmaxf(tnorm, fabsf(d[i]) + fabsf(e[i]) + (i > 0 ? fabsf(e[i - 1]) : 0.f));
  {
    // slot = t / 8 (one eigenvalue), 8 lanes evaluate 8 interior points of the interval
    const int slot = t >> 3, sub = t & 7;
    const bool active = slot < n;
    int b0 = 0, b1 = 0, kth = 0;
    float lo = 0.f, hi = 0.f;
    if (active) {
      b0 = blk_lo[slot];
      b1 = blk_hi[slot];
      kth = slot - b0;
      lo = 1e30f;
      hi = -1e30f;
      for (int i = b0; i <= b1; ++i) {
        const float r = (i > b0 ? fabsf(e[i - 1]) : 0.f) + (i < b1 ? fabsf(e[i]) : 0.f);
        lo = fminf(lo, d[i] - r);
        hi = fmaxf(hi, d[i] + r);
      }
      const float pad = 1e-6f * fmaxf(fabsf(lo), fabsf(hi)) + 1e-20f;
      lo -= pad;
      hi += pad;
    }
    for (int iter = 0; iter < 14; ++iter) {
      const float x = lo + (hi - lo) * (float)(sub + 1) / 9.f;
      const int c = active ? sturm_count(d, e2, b0, b1, x, 1e-30f) : 0;
      // new lo: largest x with count <= kth; new hi: smallest x with count >= kth + 1
      float nlo = (c <= kth) ? x : -1e30f;
      float nhi = (c >= kth + 1) ? x : 1e30f;
      for (int o = 4; o > 0; o >>= 1) {
        nlo = fmaxf(nlo, __shfl_xor_sync(0xffffffffu, nlo, o));
        nhi = fminf(nhi, __shfl_xor_sync(0xffffffffu, nhi, o));
      }
      if (nlo > lo) lo = nlo;
      if (nhi < hi) hi = nhi;
    }
    if (active && sub == 0) lam[slot] = 0.5f * (lo + hi);
  }
  __syncthreads();

  // ---- 3. eigenvectors of T by twisted factorization -------------------------------------------
  // Z (real) in the upper half of the A region; D+ and D- scratch in the lower half.
  const int zld = n + 1;                                            // padded: row-parallel solves
  float* Zr = reinterpret_cast<float*>(esm) + EH_MAXN * EH_MAXN;     // [n][zld] real, Z[i][slot]
  float* scratch = reinterpret_cast<float*>(esm);                   // 64 slots x 2n floats
  for (int idx = t; idx < n * zld; idx += EH_THREADS) Zr[idx] = 0.f;
  __syncthreads();
  for (int base = 0; base < n; base += 64) {
    const int slot = base + t;
    if (t < 64 && slot < n) {
      float* dp = scratch + (size_t)t * 2 * EH_MAXN;
      float* dm = dp + EH_MAXN;
      const int b0 = blk_lo[slot], b1 = blk_hi[slot];
      const float x = lam[slot];
      const float tiny = 1e-30f + 1e-7f * tnorm * 1e-6f;
      if (b0 == b1) {
        Zr[b0 * zld + slot] = 1.f;
      } else {
        float q = d[b0] - x;
        if (fabsf(q) < tiny) q = tiny;
        dp[b0] = q;
        for (int i = b0 + 1; i <= b1; ++i) {
          q = d[i] - x - e2[i - 1] / q;
          if (fabsf(q) < tiny) q = tiny;
          dp[i] = q;
        }
        q = d[b1] - x;
        if (fabsf(q) < tiny) q = tiny;
        dm[b1] = q;
        for (int i = b1 - 1; i >= b0; --i) {
          q = d[i] - x - e2[i] / q;
          if (fabsf(q) < tiny) q = tiny;
          dm[i] = q;
        }
        int r = b0;
        float best = 3.4e38f;
        for (int i = b0; i <= b1; ++i) {
          const float g = fabsf(dp[i] + dm[i] - (d[i] - x));
          if (g < best) {
            best = g;
            r = i;
          }
        }
        float nrm = 1.f;
        Zr[r * zld + slot] = 1.f;
        float z = 1.f;
        for (int i = r - 1; i >= b0; --i) {
          z = -(e[i] / dp[i]) * z;
          Zr[i * zld + slot] = z;
          nrm += z * z;
        }
        z = 1.f;
        for (int i = r + 1; i <= b1; ++i) {
          z = -(e[i - 1] / dm[i]) * z;
          Zr[i * zld + slot] = z;
          nrm += z * z;
        }
        const float inv = rsqrtf(nrm);
        for (int i = b0; i <= b1; ++i) Zr[i * zld + slot] *= inv;
      }
    }
    __syncthreads();
  }
  // Gram-Schmidt inside numerically degenerate clusters of a block (lam gaps <= 1e-5 |T|),
  // where twisted-factorization vectors can be nearly parallel.  One warp per block.
  for (int b = warp; b < n; b += EH_THREADS / 32) {
    if (blk_lo[b] != b) continue;
    const int b1 = blk_hi[b];
    for (int j = b + 1; j <= b1; ++j) {
      int c0 = j;
      while (c0 > b && lam[c0] - lam[c0 - 1] <= 1e-5f * tnorm) --c0;
      if (c0 == j) continue;
      for (int p = c0; p < j; ++p) {
        float s = 0.f;
        for (int i = b + lane; i <= b1; i += 32) s += Zr[i * zld + p] * Zr[i * zld + j];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        for (int i = b + lane; i <= b1; i += 32) Zr[i * zld + j] -= s * Zr[i * zld + p];
        __syncwarp();
      }
      float s = 0.f;
      for (int i = b + lane; i <= b1; i += 32) s += Zr[i * zld + j] * Zr[i * zld + j];
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      const float inv = rsqrtf(fmaxf(s, 1e-30f));
      for (int i = b + lane; i <= b1; i += 32) Zr[i * zld + j] *= inv;
      __syncwarp();
    }
  }
  __syncthreads();
  // Cholesky-QR of Z (real): G = Z^T Z = L L^T, Z <- Z L^{-T}.  Close but separated
  // eigenvalues leave Z orthogonal only to ~eps |T| / gap; this restores orthonormality
  // (G = I + O(1e-4), so L is well conditioned and the columns stay eigenvectors).
  {
    float* G = scratch;                                              // [n][n] real, lower
    for (int idx = t; idx < n * n; idx += EH_THREADS) {
      const int i = idx / n, j = idx - (idx / n) * n;
      if (j > i) continue;
      float acc = 0.f;
      for (int r = 0; r < n; ++r) acc += Zr[r * zld + i] * Zr[r * zld + j];
      G[i * n + j] = acc;
    }
    __syncthreads();
    for (int j = 0; j < n; ++j) {
      if (t == 0) G[j * n + j] = sqrtf(fmaxf(G[j * n + j], 1e-30f));
      __syncthreads();
      const float inv = 1.f / G[j * n + j];
      for (int i = j + 1 + t; i < n; i += EH_THREADS) G[i * n + j] *= inv;
      __syncthreads();
      const int mm = n - 1 - j;
      for (int idx = t; idx < mm * mm; idx += EH_THREADS) {
        const int i = j + 1 + idx / mm, k = j + 1 + idx % mm;
        if (k <= i) G[i * n + k] -= G[i * n + j] * G[k * n + j];
      }
      __syncthreads();
    }
    // row r of Z: x L^T = z  ->  x_j = (z_j - sum_{k<j} x_k L_jk) / L_jj
    if (t < n) {
      float* zrow = Zr + t * zld;
      for (int j = 0; j < n; ++j) {
        float acc = zrow[j];
        for (int k = 0; k < j; ++k) acc -= zrow[k] * G[j * n + k];
        zrow[j] = acc / G[j * n + j];
      }
    }
  }
  __syncthreads();

  // ---- 4. V = H_0 ... H_{n-2} Z ------------------------------------------------------------
  // expand Z to complex in the A region (row-major, ld = n)
  float2* V = A;
  {
    float zr[EH_MAXN * EH_MAXN / EH_THREADS];
#pragma unroll
    for (int q = 0; q < EH_MAXN * EH_MAXN / EH_THREADS; ++q) {
      const int idx = t + q * EH_THREADS;
      zr[q] = idx < n * n ? Zr[(idx / n) * zld + idx % n] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < EH_MAXN * EH_MAXN / EH_THREADS; ++q) {
      const int idx = t + q * EH_THREADS;
      if (idx < n * n) V[idx] = make_float2(zr[q], 0.f);
    }
  }
  __syncthreads();
  for (int k = n - 2; k >= 0; --k) {
    const int m = n - k - 1;
    roff -= m;
    const float2 tk = tau[k];
    if (tk.x == 0.f && tk.y == 0.f) continue;
    const float2* v = R + roff;
    // s_j = sum_i conj(v_i) V[k+1+i][j]; 8 threads per column
    {
      const int col = t >> 3, sub = t & 7;
      float2 acc = make_float2(0.f, 0.f);
      if (col < n)
        for (int i = sub; i < m; i += 8) {
          const float2 q = cmc(v[i], V[(k + 1 + i) * n + col]);
          acc.x += q.x;
          acc.y += q.y;
        }
      for (int o = 4; o > 0; o >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
      }
      if (col < n && sub == 0) wv[col] = cm(tk, acc);
    }
    __syncthreads();
    for (int idx = t; idx < m * n; idx += EH_THREADS) {
      const int i = idx / n, j = idx - (idx / n) * n;
      const float2 a = cm(v[i], wv[j]);
      float2 x = V[(k + 1 + i) * n + j];
      V[(k + 1 + i) * n + j] = make_float2(x.x - a.x, x.y - a.y);
    }
    __syncthreads();
  }
  for (int idx = t; idx < n * n; idx += EH_THREADS) {
    const float2 x = V[idx];
    Vout[idx] = make_double2((double)x.x, (double)x.y);
  }
}

}  // namespace

void eigh_householder_f32(const double2* A, double2* V, int n, cudaStream_t s) {
  if (n > EH_MAXN) fail(KS_ERR_ARG, "eigh_householder_f32: n=%d > %d", n, EH_MAXN);
  const size_t smem = ((size_t)EH_MAXN * (EH_MAXN + 1) + (size_t)EH_MAXN * (EH_MAXN - 1) / 2) * sizeof(float2);
  static bool attr = false;
  if (!attr) {
    KS_CUDA(cudaFuncSetAttribute(k_eigh_householder, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = true;
  }
  k_eigh_householder<<<1, EH_THREADS, smem, s>>>(A, n, V);
  KS_CHECK_LAUNCH();
}

}  // namespace ks
