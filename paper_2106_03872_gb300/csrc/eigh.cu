// Hermitian eigen-decomposition of the Rayleigh-Ritz matrix on the mixed path (n <= 128),
// one CTA of 1024 threads, FP32, matrix in shared memory:
//
//   1. Householder reduction A = Q T Q^H to a real symmetric tridiagonal T: for column k the
//      reflector H_k = I - tau_k v_k v_k^H (v_k[0] = 1) maps A[k+1:, k] to (beta_k, 0, ...)
//      with real beta_k; the trailing block is updated as A -= v w^H + w v^H with
//      w = tau A v - (tau/2)(w'^H v) v (the classic two-sided Hermitian update).  The update
//      of step k-1 is applied in the same pass over the trailing block as the product A v_k
//      of step k, so each step is one pass and one barrier; every warp forms v_k itself from
//      column k (identical arithmetic in every warp).
//   2. T is split where an off-diagonal element is negligible; every block's eigenvalues are
//      found by multisection on its Sturm count (8 lanes per eigenvalue, 9-way split per
//      step) until the bracket is a few ulps of |T| wide.
//   3. Eigenvectors of each block by twisted factorization (backward and forward pivots,
//      twist index at the smallest |gamma|); inside numerically degenerate clusters, inverse
//      iteration from pseudo-random starts with Gram-Schmidt against the earlier members;
//      then Newton-Schulz steps Z <- Z (3I - Z^T Z) / 2 until Z^T Z = I
//      to FP32 accuracy (close but separated eigenvalues leave twisted-factorization vectors
//      orthogonal only to ~eps |T| / gap).
//   4. Back-transformation V = H_0 H_1 ... H_{n-2} Z, each thread holding 16 rows of one
//      column of V in registers (8 threads per column).
//
// The FP32 vectors are written as complex128 columns; the caller takes the eigenvalues as
// FP64 Rayleigh quotients of these vectors on the FP64 matrix, then sorts and fixes phases.
//
// The block-iteration variant (rr_step_mixed) runs the whole Rayleigh-Ritz step of one
// iteration in the same CTA, all in FP32 with FP32 inputs and outputs (FP64 conversions run
// at the FP64 rate, which one SM cannot afford):
//   0. H_sub = conj(M) H_raw M^T from the raw projection H_raw = Psi^H (H Psi) and the
//      lower-triangular orthonormaliser M (T = H_raw M^T, then conj(M) T in place, row blocks
//      from the bottom up, since row block b of the result needs T rows <= b only);
//   1-4 as above, without the Newton-Schulz steps (the next CholQR orthonormalises);
//   5. C = Vt M and the steepest-descent step matrix Mcat = [(I + alpha Lambda) C | -alpha C]
//      with rows in ascending order of the FP32 eigenvalues.
// H_sub and the eigenvectors are exported so that ritz_values can form the reported FP64
// Rayleigh quotients off the iteration's critical path.
#include "kernels.h"

namespace ks {

namespace {

constexpr int EH_MAXN = 128;
constexpr int EH_THREADS = 1024;
constexpr int EH_WARPS = EH_THREADS / 32;
constexpr unsigned FULL = 0xffffffffu;
// shared memory: the matrix [EH_MAXN][EH_MAXN + 1], then a region for the packed reflectors
// (n(n-1)/2) that also stages operand rows in the Rayleigh-Ritz phases (64 x EH_MAXN)
constexpr int EH_AREG = EH_MAXN * (EH_MAXN + 1);
constexpr int EH_RREG = EH_MAXN * (EH_MAXN - 1) / 2 > 64 * EH_MAXN ? EH_MAXN * (EH_MAXN - 1) / 2 : 64 * EH_MAXN;
constexpr size_t EH_SMEM = (size_t)(EH_AREG + EH_RREG) * sizeof(float2);

__device__ __forceinline__ float2 cm(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ float2 cmc(float2 a, float2 b) {   // conj(a) * b
  return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 cfma(float2 acc, float2 a, float2 b) {   // acc + a b
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
  return acc;
}
__device__ __forceinline__ float2 cfmac(float2 acc, float2 a, float2 b) {  // acc + conj(a) b
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(-a.y, b.x, acc.y);
  return acc;
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 warp_sum(float2 v) {
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(FULL, v.x, o);
    v.y += __shfl_xor_sync(FULL, v.y, o);
  }
  return v;
}

// Number of eigenvalues of T[b0..b1] below x (Sturm count of the LDL^T pivots).
__device__ __forceinline__ int sturm_count(const float* d, const float* e2, int b0, int b1, float x, float pivmin) {
  int c = 0;
  float q = d[b0] - x;
  if (fabsf(q) < pivmin) q = -pivmin;
  c += q < 0.f;
  for (int i = b0 + 1; i <= b1; ++i) {
    q = d[i] - x - __fdividef(e2[i - 1], q);
    if (fabsf(q) < pivmin) q = -pivmin;
    c += q < 0.f;
  }
  return c;
}

// Phase 0 of the Rayleigh-Ritz variant: A = conj(M) H_raw M^T (FP32), Hermitian part, in the
// [n][ld] matrix region; R (EH_RREG float2) stages operand chunks.  M is lower triangular.
// Thread (warp w, lane): rows 4w + u (u < 4), columns lane + 32v (v < 4), 16 accumulators; each
// element's sum runs over k in ascending order (terms of M's zero triangle add exact zeros).
constexpr int RR_KC = 16, RR_MLD = EH_MAXN + 1;
__device__ __forceinline__ void subspace_matrix(const float2* __restrict__ Hraw, const float2* __restrict__ M, int n,
                                                float2* A, float2* R, float2* __restrict__ Aout) {
  const int ld = n + 1;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const float2 zero = make_float2(0.f, 0.f);
  float2 acc[4][4];
  // T = H_raw M^T: T_ij = sum_k H_ik M_jk
  float2* Hs = R;                                                    // [EH_MAXN][RR_KC]: H_i,k0+kk
  float2* Mt = R + EH_MAXN * RR_KC;                                  // [RR_KC][RR_MLD]: M_j,k0+kk
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = zero;
  for (int k0 = 0; k0 < n; k0 += RR_KC) {
    __syncthreads();
    for (int e = t; e < EH_MAXN * RR_KC; e += EH_THREADS) {
      const int i = e / RR_KC, k = k0 + e % RR_KC;
      Hs[e] = (i < n && k < n) ? Hraw[i * n + k] : zero;
    }
    for (int e = t; e < EH_MAXN * RR_KC; e += EH_THREADS) {
      const int j = e / RR_KC, kk = e % RR_KC, k = k0 + kk;
      Mt[kk * RR_MLD + j] = (j < n && k < n) ? M[j * n + k] : zero;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < RR_KC; ++kk) {
      float2 hv[4], mv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) hv[u] = Hs[(4 * warp + u) * RR_KC + kk];
#pragma unroll
      for (int v = 0; v < 4; ++v) mv[v] = Mt[kk * RR_MLD + lane + 32 * v];
#pragma unroll
      for (int v = 0; v < 4; ++v)
        if (32 * v + 31 >= k0)                                       // M_jk = 0 for every j of group v
#pragma unroll
          for (int u = 0; u < 4; ++u) acc[u][v] = cfma(acc[u][v], hv[u], mv[v]);
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int i = 4 * warp + u, j = lane + 32 * v;
      if (i < n && j < n) A[i * ld + j] = acc[u][v];
    }
  // A = conj(M) T: A_ij = sum_{k <= i} conj(M_ik) T_kj, all rows at once (written after the sums)
  float2* Ms = R;                                                    // [EH_MAXN][RR_KC]: M_i,k0+kk
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = zero;
  for (int k0 = 0; k0 < n; k0 += RR_KC) {
    __syncthreads();
    for (int e = t; e < EH_MAXN * RR_KC; e += EH_THREADS) {
      const int i = e / RR_KC, k = k0 + e % RR_KC;
      Ms[e] = (i < n && k < n) ? M[i * n + k] : zero;
    }
    __syncthreads();
    const int kend = min(RR_KC, n - k0);
    if (4 * warp + 3 >= k0) {                                        // M_ik = 0 for every row i of the warp
      for (int kk = 0; kk < kend; ++kk) {
        const int k = k0 + kk;
        float2 ma[4], tv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) ma[u] = Ms[(4 * warp + u) * RR_KC + kk];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int j = lane + 32 * v;
          tv[v] = j < n ? A[k * ld + j] : zero;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v] = cfmac(acc[u][v], ma[u], tv[v]);
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int i = 4 * warp + u, j = lane + 32 * v;
      if (i < n && j < n) A[i * ld + j] = acc[u][v];
    }
  __syncthreads();
  // Hermitian part (one thread per pair), real diagonal
  for (int i = warp; i < n; i += EH_WARPS)
    for (int j = lane; j <= i; j += 32) {
      const float2 a = A[i * ld + j], b = A[j * ld + i];
      const float2 h = make_float2(0.5f * (a.x + b.x), i == j ? 0.f : 0.5f * (a.y - b.y));
      A[i * ld + j] = h;
      A[j * ld + i] = make_float2(h.x, -h.y);
    }
  __syncthreads();
  for (int i = warp; i < n; i += EH_WARPS)
    for (int j = lane; j < n; j += 32) Aout[i * n + j] = A[i * ld + j];
}

// Phase 5 of the Rayleigh-Ritz variant: with V staged in the matrix region (V_kr at k ld + r),
// C = Vt M (C_rj = sum_{k >= j} V_kr M_kj, k ascending) and Mcat row rank(r) =
// [(1 + alpha lam_r) C_r | -alpha C_r].  Thread: rows r = 4w + u, columns lane + 32v.
__device__ __forceinline__ void step_matrix(const float2* Vs, const float2* __restrict__ M, int n, const float* lam,
                                            const int* rank, float alpha, float2* R, float2* __restrict__ Mcat) {
  const int ld = n + 1;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const float2 zero = make_float2(0.f, 0.f);
  float2* Ms = R;                                                    // [RR_KC][EH_MAXN]: M rows k0..
  float2 acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = zero;
  for (int k0 = 0; k0 < n; k0 += RR_KC) {
    __syncthreads();
    for (int e = t; e < RR_KC * EH_MAXN; e += EH_THREADS) {
      const int k = k0 + e / EH_MAXN, j = e % EH_MAXN;
      Ms[e] = (k < n && j < n) ? M[k * n + j] : zero;
    }
    __syncthreads();
    const int kend = min(RR_KC, n - k0);
    for (int kr = 0; kr < kend; ++kr) {
      const int k = k0 + kr;
      float2 vr[4], mv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int r = 4 * warp + u;
        vr[u] = r < n ? Vs[k * ld + r] : zero;
      }
#pragma unroll
      for (int v = 0; v < 4; ++v) mv[v] = Ms[kr * EH_MAXN + lane + 32 * v];
#pragma unroll
      for (int v = 0; v < 4; ++v)
        if (32 * v <= k)                                             // M_kj = 0 for j > k
#pragma unroll
          for (int u = 0; u < 4; ++u) acc[u][v] = cfma(acc[u][v], vr[u], mv[v]);
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int r = 4 * warp + u;
    if (r < n) {
      const float f = 1.f + alpha * lam[r];
      float2* row = Mcat + (size_t)rank[r] * 2 * n;
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const int j = lane + 32 * v;
        if (j < n) {
          row[j] = make_float2(f * acc[u][v].x, f * acc[u][v].y);
          row[n + j] = make_float2(-alpha * acc[u][v].x, -alpha * acc[u][v].y);
        }
      }
    }
  }
}

// Inputs and outputs of the Rayleigh-Ritz variant (all device pointers, row-major, FP32).
struct RRStep {
  const float2* Hraw;   // [n][n] Psi^H (H Psi)
  const float2* M;      // [n][n] lower-triangular orthonormaliser
  float alpha;          // steepest-descent step
  float2* Mcat;         // [n][2n] step matrix
  float2* Aout;         // [n][n] Hermitian subspace matrix
  float2* Vout;         // [n][n] eigenvectors, column j for lam_j (unsorted)
  int* perm;            // [n] rank of lam_j
};

template <bool RR>
__global__ void __launch_bounds__(EH_THREADS, 1)
    k_eigh_householder(const double2* __restrict__ H, int n, double2* __restrict__ Vout, RRStep rr) {
  extern __shared__ __align__(16) unsigned char esm[];
  const int ld = n + 1;
  float2* A = reinterpret_cast<float2*>(esm);                       // [n][ld]
  float2* R = A + EH_AREG;                                          // packed reflectors
  __shared__ float d[EH_MAXN], e[EH_MAXN], e2[EH_MAXN], lam[EH_MAXN];
  __shared__ float2 tau[EH_MAXN], wvp[2][EH_MAXN], red[2][EH_WARPS];
  __shared__ int blk_lo[EH_MAXN], blk_hi[EH_MAXN];
  __shared__ float s_err[EH_WARPS];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;

  if constexpr (RR) {
    subspace_matrix(rr.Hraw, rr.M, n, A, R, rr.Aout);
  } else {
    for (int idx = t; idx < n * n; idx += EH_THREADS) {
      const int i = idx / n, j = idx - (idx / n) * n;
      const double2 h = H[idx];
      A[i * ld + j] = make_float2((float)h.x, i == j ? 0.f : (float)h.y);
    }
  }
  __syncthreads();

  // ---- 1. tridiagonalization ---------------------------------------------------------------
  // Entering step k, A[k:, k:] holds the updates of steps < k-1; the update of step k-1
  // (v_{k-1} at R + rprev, w_{k-1} = wvp[(k-1)&1] + ap v_{k-1}) is still to be applied.
  // Lane-owned indices: rows / columns k+1+lane+32q, q < 4.
  int rprev = 0, roff = 0;
  for (int k = 0; k + 1 < n; ++k) {
    const int m = n - k - 1;
    const bool hp = k > 0;
    const int pb = (k + 1) & 1;                                     // buffer of step k-1
    float2 ap = make_float2(0.f, 0.f);
    if (hp) {
      const float2 s = warp_sum(red[pb][lane]);
      const float2 h = cm(tau[k - 1], s);
      ap = make_float2(-0.5f * h.x, -0.5f * h.y);
    }
    // pending-update vectors at the lane's indices and at k
    float2 vp[4], wp[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = k + 1 + lane + 32 * q;
      vp[q] = make_float2(0.f, 0.f);
      wp[q] = make_float2(0.f, 0.f);
      if (hp && j < n) {
        vp[q] = R[rprev + j - k];
        wp[q] = cadd(wvp[pb][j], cm(ap, vp[q]));
      }
    }
    const float2 wk = hp ? cadd(wvp[pb][k], ap) : make_float2(0.f, 0.f);   // v_{k-1}[k] = 1
    // column k after the pending update: x_i = A_ik - (v_i conj(w_k) + w_i)
    float2 x[4];
    float xn2 = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = k + 1 + lane + 32 * q;
      x[q] = make_float2(0.f, 0.f);
      if (i < n) {
        const float2 a = A[i * ld + k];
        const float2 u = cadd(make_float2(vp[q].x * wk.x + vp[q].y * wk.y, vp[q].y * wk.x - vp[q].x * wk.y), wp[q]);
        x[q] = csub(a, u);
        if (q > 0 || lane > 0) xn2 += x[q].x * x[q].x + x[q].y * x[q].y;
      }
    }
    for (int o = 16; o > 0; o >>= 1) xn2 += __shfl_xor_sync(FULL, xn2, o);
    const float2 al = make_float2(__shfl_sync(FULL, x[0].x, 0), __shfl_sync(FULL, x[0].y, 0));
    float2 tk, sc = make_float2(0.f, 0.f);
    float ek;
    const float s2 = al.x * al.x + al.y * al.y + xn2;
    if (xn2 == 0.f && al.y == 0.f) {
      tk = make_float2(0.f, 0.f);
      ek = al.x;
    } else if (s2 < 1e-30f) {
      // a column already reduced up to rounding noise (|x| < 1e-15): no reflection and a zero
      // off-diagonal element, which moves eigenvalues by < 1e-15; forming the reflector from
      // such a column would underflow its squares and divide by zero
      tk = make_float2(0.f, 0.f);
      ek = 0.f;
    } else {
      const float beta = -copysignf(sqrtf(al.x * al.x + al.y * al.y + xn2), al.x);
      const float rb = __frcp_rn(beta);
      tk = make_float2((beta - al.x) * rb, -al.y * rb);
      const float2 dn = make_float2(al.x - beta, al.y);            // 1 / (alpha - beta)
      const float inv = __frcp_rn(dn.x * dn.x + dn.y * dn.y);
      sc = make_float2(dn.x * inv, -dn.y * inv);
      ek = beta;
    }
    float2 vk[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = k + 1 + lane + 32 * q;
      vk[q] = (q == 0 && lane == 0) ? make_float2(1.f, 0.f) : (i < n ? cm(x[q], sc) : make_float2(0.f, 0.f));
    }
    if (warp == 0) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = k + 1 + lane + 32 * q;
        if (i < n) R[roff + i - k - 1] = vk[q];
      }
      if (lane == 0) {
        tau[k] = tk;
        e[k] = ek;
        d[k] = A[k * ld + k].x - 2.f * wk.x;
      }
    }
    // trailing block: apply the update of step k-1, then w'_i = tau_k sum_j A_ij v_j; the
    // four rows' sums are reduced together so their shuffle latencies overlap
    float2 acc[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int i = k + 1 + warp + 32 * r;
      acc[r] = make_float2(0.f, 0.f);
      if (i < n) {                                                   // warp-uniform
        float2 vi = make_float2(0.f, 0.f), wi = make_float2(0.f, 0.f);
        if (hp) {
          vi = R[rprev + i - k];
          wi = cadd(wvp[pb][i], cm(ap, vi));
        }
        float2* arow = A + i * ld;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int j = k + 1 + lane + 32 * q;
          if (j < n) {
            float2 a = arow[j];
            if (hp) {
              // v_i conj(w_j) + w_i conj(v_j)
              a.x -= (vi.x * wp[q].x + vi.y * wp[q].y) + (wi.x * vp[q].x + wi.y * vp[q].y);
              a.y -= (vi.y * wp[q].x - vi.x * wp[q].y) + (wi.y * vp[q].x - wi.x * vp[q].y);
            }
            if (i == j) a.y = 0.f;
            arow[j] = a;
            acc[r].x += a.x * vk[q].x - a.y * vk[q].y;
            acc[r].y += a.x * vk[q].y + a.y * vk[q].x;
          }
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        acc[r].x += __shfl_xor_sync(FULL, acc[r].x, o);
        acc[r].y += __shfl_xor_sync(FULL, acc[r].y, o);
      }
    float2 pw = make_float2(0.f, 0.f);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int i = k + 1 + warp + 32 * r;
      // v_k at row i lives in lane (i - k - 1) & 31 = warp, slot r
      const float2 vr = make_float2(__shfl_sync(FULL, vk[r].x, warp), __shfl_sync(FULL, vk[r].y, warp));
      if (i < n) {
        const float2 w = cm(tk, acc[r]);
        if (lane == 0) wvp[k & 1][i] = w;
        const float2 c = cmc(w, vr);
        pw.x += c.x;
        pw.y += c.y;
      }
    }
    if (lane == 0) red[k & 1][warp] = pw;
    rprev = roff;
    roff += m;
    __syncthreads();
  }
  if (t == 0) {
    if (n >= 2) {
      // last pending update (v_{n-2} = (1)), then d_{n-1}
      float2 s = make_float2(0.f, 0.f);
      for (int w = 0; w < EH_WARPS; ++w) s = cadd(s, red[n & 1][w]);
      const float2 h = cm(tau[n - 2], s);
      const float wl = wvp[n & 1][n - 1].x - 0.5f * h.x;
      d[n - 1] = A[(n - 1) * ld + (n - 1)].x - 2.f * wl;
    } else {
      d[0] = A[0].x;
    }
    e[n - 1] = 0.f;
  }
  __syncthreads();

  // ---- 2. split and eigenvalues ------------------------------------------------------------
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
  float tnorm = 0.f;
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
    const float width = 4.8e-7f * tnorm + 1e-30f;                    // ~4 ulps of |T|
    for (int iter = 0; iter < 24; ++iter) {
      const bool need = active && (hi - lo > width);
      if (!__any_sync(FULL, need)) break;
      const float x = lo + (hi - lo) * (float)(sub + 1) * (1.f / 9.f);
      const int c = need ? sturm_count(d, e2, b0, b1, x, 1e-30f) : 0;
      // new lo: largest x with count <= kth; new hi: smallest x with count >= kth + 1
      float nlo = (need && c <= kth) ? x : -1e30f;
      float nhi = (need && c >= kth + 1) ? x : 1e30f;
      for (int o = 4; o > 0; o >>= 1) {
        nlo = fmaxf(nlo, __shfl_xor_sync(FULL, nlo, o));
        nhi = fminf(nhi, __shfl_xor_sync(FULL, nhi, o));
      }
      if (nlo > lo) lo = nlo;
      if (nhi < hi) hi = nhi;
    }
    if (active && sub == 0) lam[slot] = 0.5f * (lo + hi);
  }
  __syncthreads();

  // ---- 3. eigenvectors of T ----------------------------------------------------------------
  // Z (real, [n][zld]) in the upper half of the A region; D- pivots [n][n] and later
  // Z^T Z in the lower half.
  const int zld = n + 1;
  const float tiny = 1e-30f + 1e-13f * tnorm;                        // pivot floor
  float* Zr = reinterpret_cast<float*>(esm) + EH_MAXN * EH_MAXN;
  float* low = reinterpret_cast<float*>(esm);
  for (int idx = t; idx < n * zld; idx += EH_THREADS) Zr[idx] = 0.f;
  __syncthreads();
  if (t < n) {
    const int slot = t;
    const int b0 = blk_lo[slot], b1 = blk_hi[slot];
    const float x = lam[slot];
    if (b0 == b1) {
      Zr[b0 * zld + slot] = 1.f;
    } else {
      // backward pivots D-: dm_i = d_i - x - e_i^2 / dm_{i+1}, kept in low[i][slot]
      float q = d[b1] - x;
      if (fabsf(q) < tiny) q = tiny;
      low[b1 * n + slot] = q;
      for (int i = b1 - 1; i >= b0; --i) {
        q = d[i] - x - __fdividef(e2[i], q);
        if (fabsf(q) < tiny) q = tiny;
        low[i * n + slot] = q;
      }
      // forward pivots D+ with gamma_i = dp_i + dm_i - (d_i - x); the ratios -e_i / dp_i
      // go to Z's column until the twist index r (argmin |gamma|) is known
      int r = b0;
      float best = 3.4e38f;
      q = d[b0] - x;
      if (fabsf(q) < tiny) q = tiny;
      for (int i = b0; i <= b1; ++i) {
        if (i > b0) {
          q = d[i] - x - __fdividef(e2[i - 1], q);
          if (fabsf(q) < tiny) q = tiny;
        }
        const float g = fabsf(q + low[i * n + slot] - (d[i] - x));
        if (g < best) {
          best = g;
          r = i;
        }
        if (i < b1) Zr[i * zld + slot] = -__fdividef(e[i], q);
      }
      float nrm = 1.f, z = 1.f;
      for (int i = r - 1; i >= b0; --i) {
        z *= Zr[i * zld + slot];
        Zr[i * zld + slot] = z;
        nrm += z * z;
      }
      Zr[r * zld + slot] = 1.f;
      z = 1.f;
      for (int i = r + 1; i <= b1; ++i) {
        z *= -__fdividef(e[i - 1], low[i * n + slot]);
        Zr[i * zld + slot] = z;
        nrm += z * z;
      }
      const float inv = rsqrtf(nrm);
      for (int i = b0; i <= b1; ++i) Zr[i * zld + slot] *= inv;
    }
  }
  __syncthreads();
  // Degenerate clusters of a block (lam gaps <= 1e-5 |T|): twisted factorization returns
  // (nearly) the same vector for every member, so each member after the first is recomputed
  // by inverse iteration -- two LDL^T solves of (T - lam_j) y = x from a pseudo-random start,
  // each followed by Gram-Schmidt against the earlier members of the cluster (the scheme of
  // LAPACK's stein).  One warp per block; lane 0 runs the serial solves.
  for (int b = warp; b < n; b += EH_WARPS) {
    if (blk_lo[b] != b) continue;
    const int b1 = blk_hi[b];
    float* Lc = low + warp * EH_MAXN;                                // L's subdiagonal
    for (int j = b + 1; j <= b1; ++j) {
      int c0 = j;
      while (c0 > b && lam[c0] - lam[c0 - 1] <= 1e-5f * tnorm) --c0;
      if (c0 == j) continue;
      for (int i = b + lane; i <= b1; i += 32) {
        const unsigned hsh = (unsigned)(i * 131 + j * 7919) * 2654435761u;
        Zr[i * zld + j] = (float)(hsh >> 16) * (1.f / 32768.f) - 1.f;
      }
      __syncwarp();
      const float lj = lam[j];
      for (int it = 0; it < 2; ++it) {
        if (lane == 0) {
          float piv = d[b] - lj;
          if (fabsf(piv) < tiny) piv = tiny;
          float u = Zr[b * zld + j];
          Zr[b * zld + j] = __fdividef(u, piv);
          for (int i = b + 1; i <= b1; ++i) {
            const float l = __fdividef(e[i - 1], piv);
            Lc[i - 1] = l;
            piv = d[i] - lj - l * e[i - 1];
            if (fabsf(piv) < tiny) piv = tiny;
            u = Zr[i * zld + j] - l * u;
            Zr[i * zld + j] = __fdividef(u, piv);
          }
          for (int i = b1 - 1; i >= b; --i) Zr[i * zld + j] -= Lc[i] * Zr[(i + 1) * zld + j];
        }
        __syncwarp();
        for (int p = c0; p < j; ++p) {
          float sd = 0.f;
          for (int i = b + lane; i <= b1; i += 32) sd += Zr[i * zld + p] * Zr[i * zld + j];
          for (int o = 16; o > 0; o >>= 1) sd += __shfl_xor_sync(FULL, sd, o);
          for (int i = b + lane; i <= b1; i += 32) Zr[i * zld + j] -= sd * Zr[i * zld + p];
          __syncwarp();
        }
        float sn = 0.f;
        for (int i = b + lane; i <= b1; i += 32) sn += Zr[i * zld + j] * Zr[i * zld + j];
        for (int o = 16; o > 0; o >>= 1) sn += __shfl_xor_sync(FULL, sn, o);
        const float inv = rsqrtf(fmaxf(sn, 1e-30f));
        for (int i = b + lane; i <= b1; i += 32) Zr[i * zld + j] *= inv;
        __syncwarp();
      }
    }
  }
  __syncthreads();
  // Newton-Schulz: G = Z^T Z; while max |G - I| > 2e-6: Z <- 1.5 Z - 0.5 Z G.
  // Thread tiles: rows warp + 32u, columns lane + 32v (u, v < 4).  The Rayleigh-Ritz variant
  // skips it: its vectors only span the next iterate, whose CholQR orthonormalises the block,
  // and outside degenerate clusters (handled above) they are orthogonal to eps |T| / gap
  // <= 6e-3, a condition number of the step matrix within 1.01.
  if constexpr (!RR) {
    float* G = low;                                                  // [n][n]
    for (int it = 0; it < 4; ++it) {
      float g[4][4] = {};
      for (int i = 0; i < n; ++i) {
        float za[4], zb[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int a = warp + 32 * u, b = lane + 32 * u;
          za[u] = a < n ? Zr[i * zld + a] : 0.f;
          zb[u] = b < n ? Zr[i * zld + b] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) g[u][v] += za[u] * zb[v];
      }
      float err = 0.f;
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int a = warp + 32 * u, b = lane + 32 * v;
          if (a < n && b < n) {
            G[a * n + b] = g[u][v];
            err = fmaxf(err, fabsf(g[u][v] - (a == b ? 1.f : 0.f)));
          }
        }
      for (int o = 16; o > 0; o >>= 1) err = fmaxf(err, __shfl_xor_sync(FULL, err, o));
      if (lane == 0) s_err[warp] = err;
      __syncthreads();
      float emax = 0.f;
      for (int w = 0; w < EH_WARPS; ++w) emax = fmaxf(emax, s_err[w]);
      if (!(emax > 2e-6f)) break;                                    // uniform
      float z[4][4] = {};
      for (int b = 0; b < n; ++b) {
        float zr[4], gb[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = warp + 32 * u, a = lane + 32 * u;
          zr[u] = i < n ? Zr[i * zld + b] : 0.f;
          gb[u] = a < n ? G[b * n + a] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) z[u][v] += zr[u] * gb[v];
      }
      __syncthreads();
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int i = warp + 32 * u, a = lane + 32 * v;
          if (i < n && a < n) Zr[i * zld + a] = 1.5f * Zr[i * zld + a] - 0.5f * z[u][v];
        }
      __syncthreads();
    }
  }

  // ---- 4. V = H_0 ... H_{n-2} Z ------------------------------------------------------------
  // thread (column j = t / 8, s = t % 8) holds rows s + 8p, p < 16.  The reflectors are
  // expanded into a zero-padded [n-1][EH_MAXN] layout in the A region (v_k[i] = 0 for i <= k
  // and i >= n), so no row needs a bounds test.
  {
    const int j = t >> 3, s = t & 7;
    float2 V[16];
#pragma unroll
    for (int p = 0; p < 16; ++p) {
      const int i = s + 8 * p;
      V[p] = make_float2((i < n && j < n) ? Zr[i * zld + j] : 0.f, 0.f);
    }
    __syncthreads();
    float2* Rf = A;
    for (int idx = t; idx < (n - 1) * EH_MAXN; idx += EH_THREADS) {
      const int k = idx / EH_MAXN, i = idx - k * EH_MAXN;
      const int ro = k * (n - 1) - (k * (k - 1)) / 2;
      Rf[idx] = (i > k && i < n) ? R[ro + i - k - 1] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int k = n - 2; k >= 0; --k) {
      const float2 tk = tau[k];
      if (tk.x == 0.f && tk.y == 0.f) continue;                      // uniform
      const float2* v = Rf + k * EH_MAXN + s;                        // v[8p] = v_k at row s + 8p
      const int pskip = (k + 1) >> 3;                                // rows s + 8p < k+1 below
      float2 dot = make_float2(0.f, 0.f);
#pragma unroll
      for (int p = 0; p < 16; ++p) {
        if (p >= pskip) {
          const float2 c = cmc(v[8 * p], V[p]);
          dot.x += c.x;
          dot.y += c.y;
        }
      }
      for (int o = 4; o > 0; o >>= 1) {
        dot.x += __shfl_xor_sync(FULL, dot.x, o);
        dot.y += __shfl_xor_sync(FULL, dot.y, o);
      }
      const float2 c = cm(tk, dot);
#pragma unroll
      for (int p = 0; p < 16; ++p)
        if (p >= pskip) V[p] = csub(V[p], cm(v[8 * p], c));
    }
    // stage through shared memory (the A region) for coalesced complex128 stores
    __syncthreads();
    float2* Vs = A;                                                  // [n][ld]
    if (j < n) {
#pragma unroll
      for (int p = 0; p < 16; ++p) {
        const int i = s + 8 * p;
        if (i < n) Vs[i * ld + j] = V[p];
      }
    }
  }
  __syncthreads();
  if constexpr (RR) {
    // ranks of the eigenvalues (ties by index) and the exported vectors
    int* rank = blk_lo;
    if (t < n) {
      const float li = lam[t];
      int r = 0;
      for (int j = 0; j < n; ++j) r += (lam[j] < li) || (lam[j] == li && j < t);
      rank[t] = r;
      rr.perm[t] = r;
    }
    for (int i = warp; i < n; i += EH_WARPS)
      for (int j = lane; j < n; j += 32) rr.Vout[i * n + j] = A[i * ld + j];
    __syncthreads();
    step_matrix(A, rr.M, n, lam, rank, rr.alpha, R, rr.Mcat);
  } else {
    for (int idx = t; idx < n * n; idx += EH_THREADS) {
      const int i = idx / n, j = idx - (idx / n) * n;
      const float2 v = A[i * ld + j];
      Vout[idx] = make_double2((double)v.x, (double)v.y);
    }
  }
}

// Reported eigenvalues of the Rayleigh-Ritz variant: FP64 Rayleigh quotients of the FP32
// eigenvectors on the FP32 subspace matrix, eig[perm[j]] = Re(v_j^H A v_j) / (v_j^H v_j).
__global__ void k_ritz_values(const float2* __restrict__ A, const float2* __restrict__ V, const int* __restrict__ perm,
                              int n, double* __restrict__ eig) {
  const int j = blockIdx.x;
  __shared__ double2 v[EH_MAXN];
  __shared__ double red[2][8];
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const float2 x = V[k * n + j];
    v[k] = make_double2((double)x.x, (double)x.y);
  }
  __syncthreads();
  double num = 0.0, den = 0.0;
  for (int a = threadIdx.x >> 5; a < n; a += blockDim.x >> 5) {
    const double2 va = v[a];
    double2 s = make_double2(0.0, 0.0);
    for (int b = threadIdx.x & 31; b < n; b += 32) {
      const float2 h = A[a * n + b];
      const double2 vb = v[b];
      s.x += (double)h.x * vb.x - (double)h.y * vb.y;
      s.y += (double)h.x * vb.y + (double)h.y * vb.x;
    }
    num += va.x * s.x + va.y * s.y;                                  // Re(conj(v_a) s)
    if ((threadIdx.x & 31) == 0) den += va.x * va.x + va.y * va.y;
  }
  for (int o = 16; o > 0; o >>= 1) {
    num += __shfl_xor_sync(FULL, num, o);
    den += __shfl_xor_sync(FULL, den, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = num;
    red[1][threadIdx.x >> 5] = den;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a += red[0][w];
      b += red[1][w];
    }
    eig[perm[j]] = a / b;
  }
}

}  // namespace

void eigh_householder_f32(const double2* A, double2* V, int n, cudaStream_t s) {
  if (n > EH_MAXN || n < 1) fail(KS_ERR_ARG, "eigh_householder_f32: n=%d not in [1, %d]", n, EH_MAXN);
  static bool attr = false;
  if (!attr) {
    KS_CUDA(cudaFuncSetAttribute(k_eigh_householder<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)EH_SMEM));
    attr = true;
  }
  k_eigh_householder<false><<<1, EH_THREADS, EH_SMEM, s>>>(A, n, V, RRStep{});
  KS_CHECK_LAUNCH();
}

void rr_step_mixed(const float2* Hraw, const float2* M, double alpha, int n, float2* Mcat, float2* Aout,
                   float2* Vout, int* perm, cudaStream_t s) {
  if (n > EH_MAXN || n < 1) fail(KS_ERR_ARG, "rr_step_mixed: n=%d not in [1, %d]", n, EH_MAXN);
  static bool attr = false;
  if (!attr) {
    KS_CUDA(cudaFuncSetAttribute(k_eigh_householder<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)EH_SMEM));
    attr = true;
  }
  const RRStep rr{Hraw, M, (float)alpha, Mcat, Aout, Vout, perm};
  k_eigh_householder<true><<<1, EH_THREADS, EH_SMEM, s>>>(nullptr, n, nullptr, rr);
  KS_CHECK_LAUNCH();
}

void ritz_values(const float2* A, const float2* V, const int* perm, int n, double* eig, cudaStream_t s) {
  if (n > EH_MAXN || n < 1) fail(KS_ERR_ARG, "ritz_values: n=%d not in [1, %d]", n, EH_MAXN);
  k_ritz_values<<<n, 256, 0, s>>>(A, V, perm, n, eig);
  KS_CHECK_LAUNCH();
}

}  // namespace ks
