// Device FFT building blocks: small DFTs in registers and Stockham auto-sort stages on
// lines held in shared memory.  Lengths N = 2^a 3^b; the transform is unnormalised with
// exponent sign `sign` (+1: G -> r, -1: r -> G).
#pragma once

#include "common.h"

namespace ks {

struct FftPlan {
  int nstages;
  int radix[12];
};

inline FftPlan make_plan(int N) {
  FftPlan p{};
  int n = N;
  while (n % 4 == 0) { p.radix[p.nstages++] = 4; n /= 4; }
  while (n % 2 == 0) { p.radix[p.nstages++] = 2; n /= 2; }
  while (n % 3 == 0) { p.radix[p.nstages++] = 3; n /= 3; }
  return p;
}

// i * z
template <typename C> __device__ __forceinline__ C mul_i(C z) { return mk<C>(-z.y, z.x); }

template <int R, typename C> struct SmallDft;

template <typename C> struct SmallDft<2, C> {
  static __device__ __forceinline__ void run(C* v, int) {
    const C a = v[0], b = v[1];
    v[0] = a + b;
    v[1] = a - b;
  }
};

template <typename C> struct SmallDft<3, C> {
  static __device__ __forceinline__ void run(C* v, int sign) {
    using R = decltype(C::x);
    const R half = R(0.5);
    const R s3 = R(0.86602540378443864676) * R(sign);   // sign * sqrt(3)/2
    const C t1 = v[1] + v[2];
    const C t2 = v[1] - v[2];
    const C m = v[0] - t1 * half;
    const C r = mul_i(t2) * s3;
    v[0] = v[0] + t1;
    v[1] = m + r;
    v[2] = m - r;
  }
};

template <typename C> struct SmallDft<4, C> {
  static __device__ __forceinline__ void run(C* v, int sign) {
    const C t0 = v[0] + v[2];
    const C t1 = v[0] - v[2];
    const C t2 = v[1] + v[3];
    C t3 = mul_i(v[1] - v[3]);
    if (sign < 0) t3 = mk<C>(-t3.x, -t3.y);
    v[0] = t0 + t2;
    v[2] = t0 - t2;
    v[1] = t1 + t3;
    v[3] = t1 - t3;
  }
};

// One Stockham stage of radix R over `lines` lines of length N stored at s + l*ld.
// Ns = product of the radices already applied.  Each thread keeps up to Q butterflies in
// registers; every read happens before the barrier and every write after it, so the
// stage runs in place.  tw[t] = exp(sign 2 pi i t / N).
template <int R, int Q, typename C>
__device__ __forceinline__ void stockham_stage(C* s, int lines, int ld, int N, int Ns, const C* tw, int sign) {
  const int M = N / R;
  const int jobs = lines * M;
  const int step = N / (Ns * R);
  C v[Q][R];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int job = threadIdx.x + q * blockDim.x;
    if (job < jobs) {
      const int l = job / M, j = job - (job / M) * M;
      const int k = j % Ns;
      const C* line = s + l * ld;
#pragma unroll
      for (int r = 0; r < R; ++r) v[q][r] = line[j + r * M];
      if (Ns > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) v[q][r] = cmul(v[q][r], tw[k * r * step]);
      }
      SmallDft<R, C>::run(v[q], sign);
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int job = threadIdx.x + q * blockDim.x;
    if (job < jobs) {
      const int l = job / M, j = job - (job / M) * M;
      const int k = j % Ns;
      C* line = s + l * ld;
      const int base = (j / Ns) * Ns * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) line[base + r * Ns] = v[q][r];
    }
  }
  __syncthreads();
}

// Full FFT of `lines` lines in shared memory.  Requires lines * N <= LINE_ELEMS and
// blockDim.x == LINE_THREADS (so every stage fits the per-thread register budget).
constexpr int LINE_THREADS = 256;
constexpr int LINE_ELEMS = 2048;

template <typename C>
__device__ __forceinline__ void fft_lines_smem(C* s, int lines, int ld, int N, const FftPlan& plan, const C* tw,
                                               int sign) {
  int Ns = 1;
  for (int i = 0; i < plan.nstages; ++i) {
    const int R = plan.radix[i];
    if (R == 4)
      stockham_stage<4, LINE_ELEMS / 4 / LINE_THREADS, C>(s, lines, ld, N, Ns, tw, sign);
    else if (R == 2)
      stockham_stage<2, LINE_ELEMS / 2 / LINE_THREADS, C>(s, lines, ld, N, Ns, tw, sign);
    else
      stockham_stage<3, (LINE_ELEMS / 3 + LINE_THREADS - 1) / LINE_THREADS, C>(s, lines, ld, N, Ns, tw, sign);
    Ns *= R;
  }
}

}  // namespace ks
