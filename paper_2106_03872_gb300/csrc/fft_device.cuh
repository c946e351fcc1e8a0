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

// ---------------------------------------------------------------------------------------------
// Generalised stages for the fused kernels: line l, element k at s[l*lstride + k*kstride];
// radices 8, 4, 2, 3; THREADS threads; one call transforms up to CAP elements (lines * N).
// LINE_FAST maps consecutive threads to consecutive lines (for lines that are columns of a
// row-major plane, so that shared-memory accesses of a warp are contiguous).
// The twiddle table holds exp(+2 pi i t/N); sign < 0 conjugates it on the fly.
// ---------------------------------------------------------------------------------------------
namespace ks {

inline FftPlan make_plan8(int N) {
  FftPlan p{};
  int n = N;
  while (n % 8 == 0) { p.radix[p.nstages++] = 8; n /= 8; }
  while (n % 4 == 0) { p.radix[p.nstages++] = 4; n /= 4; }
  while (n % 2 == 0) { p.radix[p.nstages++] = 2; n /= 2; }
  while (n % 3 == 0) { p.radix[p.nstages++] = 3; n /= 3; }
  return p;
}

template <typename C> struct SmallDft<8, C> {
  static __device__ __forceinline__ void run(C* v, int sign) {
    using R = decltype(C::x);
    const R h = R(0.70710678118654752440);
    const R sg = R(sign);
    C a[4], b[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      a[r] = v[r] + v[r + 4];
      b[r] = v[r] - v[r + 4];
    }
    // b_r *= w^r, w = exp(sign i pi/4)
    {
      const C z = b[1];
      b[1] = mk<C>(h * (z.x - sg * z.y), h * (z.y + sg * z.x));
    }
    {
      const C z = b[2];
      b[2] = mk<C>(-sg * z.y, sg * z.x);
    }
    {
      const C z = b[3];
      b[3] = mk<C>(h * (-z.x - sg * z.y), h * (-z.y + sg * z.x));
    }
    SmallDft<4, C>::run(a, sign);
    SmallDft<4, C>::run(b, sign);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      v[2 * m] = a[m];
      v[2 * m + 1] = b[m];
    }
  }
};

template <int R, int Q, int THREADS, bool LINE_FAST, typename C>
__device__ __forceinline__ void stage_g(C* s, int lines, int lstride, int kstride, int N, int Ns, const C* tw,
                                        int sign) {
  const int M = N / R;
  const int jobs = lines * M;
  const int step = N / (Ns * R);
  C v[Q][R];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int job = threadIdx.x + q * THREADS;
    if (job < jobs) {
      int l, j;
      if (LINE_FAST) {
        j = job / lines;
        l = job - j * lines;
      } else {
        l = job / M;
        j = job - l * M;
      }
      const int k = j % Ns;
      const C* line = s + l * lstride;
#pragma unroll
      for (int r = 0; r < R; ++r) v[q][r] = line[(j + r * M) * kstride];
      if (Ns > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          C w = tw[k * r * step];
          if (sign < 0) w.y = -w.y;
          v[q][r] = cmul(v[q][r], w);
        }
      }
      SmallDft<R, C>::run(v[q], sign);
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int job = threadIdx.x + q * THREADS;
    if (job < jobs) {
      int l, j;
      if (LINE_FAST) {
        j = job / lines;
        l = job - j * lines;
      } else {
        l = job / M;
        j = job - l * M;
      }
      const int k = j % Ns;
      C* line = s + l * lstride;
      const int base = (j / Ns) * Ns * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) line[(base + r * Ns) * kstride] = v[q][r];
    }
  }
  __syncthreads();
}

template <int THREADS, int CAP, bool LINE_FAST, typename C>
__device__ __forceinline__ void fft_lines_g(C* s, int lines, int lstride, int kstride, int N, const FftPlan& plan,
                                            const C* tw, int sign) {
  int Ns = 1;
  for (int i = 0; i < plan.nstages; ++i) {
    const int R = plan.radix[i];
    if (R == 8)
      stage_g<8, (CAP / 8 + THREADS - 1) / THREADS, THREADS, LINE_FAST, C>(s, lines, lstride, kstride, N, Ns, tw, sign);
    else if (R == 4)
      stage_g<4, (CAP / 4 + THREADS - 1) / THREADS, THREADS, LINE_FAST, C>(s, lines, lstride, kstride, N, Ns, tw, sign);
    else if (R == 2)
      stage_g<2, (CAP / 2 + THREADS - 1) / THREADS, THREADS, LINE_FAST, C>(s, lines, lstride, kstride, N, Ns, tw, sign);
    else
      stage_g<3, (CAP / 3 + THREADS - 1) / THREADS, THREADS, LINE_FAST, C>(s, lines, lstride, kstride, N, Ns, tw, sign);
    Ns *= R;
  }
}

// Transform `lines` lines in groups that fit CAP elements per call.
template <int THREADS, int CAP, bool LINE_FAST, typename C>
__device__ __forceinline__ void fft_lines_grouped(C* s, int lines, int lstride, int kstride, int N,
                                                  const FftPlan& plan, const C* tw, int sign) {
  const int per = CAP / N;
  for (int l0 = 0; l0 < lines; l0 += per) {
    const int nl = min(per, lines - l0);
    fft_lines_g<THREADS, CAP, LINE_FAST, C>(s + l0 * lstride, nl, lstride, kstride, N, plan, tw, sign);
  }
}

}  // namespace ks

// ---------------------------------------------------------------------------------------------
// Compile-time plans (fused kernels): N, the radix sequence (8, then 4, 2, 3), the job
// decomposition and the exponent sign are constants, so index arithmetic folds away.
// ---------------------------------------------------------------------------------------------
namespace ks {

template <int N, int Ns> struct RadixOf {
  static constexpr int rem = N / Ns;
  static constexpr int R = (rem % 8 == 0) ? 8 : (rem % 4 == 0) ? 4 : (rem % 2 == 0) ? 2 : 3;
};

// One stage over `lines` lines (<= LPC lines; LPC = lines per call).  LINE_FAST: job =
// j * LPC + l (consecutive threads on consecutive lines), else job = l * M + j.
template <int N, int Ns, int R, int THREADS, int LPC, bool LINE_FAST, int SIGN>
__device__ __forceinline__ void cstage(float2* s, int lines, int lstride, int kstride, const float2* tw) {
  constexpr int M = N / R;
  constexpr int step = N / (Ns * R);
  constexpr int JOBS = LPC * M;
  constexpr int Q = (JOBS + THREADS - 1) / THREADS;
  float2 v[Q][R];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int job = threadIdx.x + q * THREADS;
    int l, j;
    if (LINE_FAST) {
      j = job / LPC;
      l = job - j * LPC;
    } else {
      l = job / M;
      j = job - l * M;
    }
    if (job < JOBS && l < lines) {
      const int k = j % Ns;
      const float2* line = s + l * lstride;
#pragma unroll
      for (int r = 0; r < R; ++r) v[q][r] = line[(j + r * M) * kstride];
      if (Ns > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          float2 w = tw[k * r * step];
          if (SIGN < 0) w.y = -w.y;
          v[q][r] = cmul(v[q][r], w);
        }
      }
      SmallDft<R, float2>::run(v[q], SIGN);
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int job = threadIdx.x + q * THREADS;
    int l, j;
    if (LINE_FAST) {
      j = job / LPC;
      l = job - j * LPC;
    } else {
      l = job / M;
      j = job - l * M;
    }
    if (job < JOBS && l < lines) {
      const int k = j % Ns;
      float2* line = s + l * lstride;
      const int base = (j / Ns) * Ns * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) line[(base + r * Ns) * kstride] = v[q][r];
    }
  }
  __syncthreads();
}

template <int N, int Ns, int THREADS, int LPC, bool LINE_FAST, int SIGN> struct CFft {
  static __device__ __forceinline__ void run(float2* s, int lines, int lstride, int kstride, const float2* tw) {
    constexpr int R = RadixOf<N, Ns>::R;
    cstage<N, Ns, R, THREADS, LPC, LINE_FAST, SIGN>(s, lines, lstride, kstride, tw);
    CFft<N, Ns * R, THREADS, LPC, LINE_FAST, SIGN>::run(s, lines, lstride, kstride, tw);
  }
};
template <int N, int THREADS, int LPC, bool LINE_FAST, int SIGN> struct CFft<N, N, THREADS, LPC, LINE_FAST, SIGN> {
  static __device__ __forceinline__ void run(float2*, int, int, int, const float2*) {}
};

// All `lines` lines, LPC at a time.
template <int N, int THREADS, int LPC, bool LINE_FAST, int SIGN>
__device__ __forceinline__ void cfft_lines(float2* s, int lines, int lstride, int kstride, const float2* tw) {
  for (int l0 = 0; l0 < lines; l0 += LPC)
    CFft<N, 1, THREADS, LPC, LINE_FAST, SIGN>::run(s + l0 * lstride, min(LPC, lines - l0), lstride, kstride, tw);
}

}  // namespace ks
