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

// cos(2 pi m / N) for the composite in-register DFTs (N = 12, 16).
__host__ __device__ constexpr double cos_frac(int m, int N) {
  if (N == 16) {
    switch (((m % 16) + 16) % 16) {
      case 0: return 1.0;
      case 1: case 15: return 0.92387953251128675613;
      case 2: case 14: return 0.70710678118654752440;
      case 3: case 13: return 0.38268343236508977173;
      case 4: case 12: return 0.0;
      case 5: case 11: return -0.38268343236508977173;
      case 6: case 10: return -0.70710678118654752440;
      case 7: case 9: return -0.92387953251128675613;
      default: return -1.0;
    }
  }
  switch (((m % 12) + 12) % 12) {
    case 0: return 1.0;
    case 1: case 11: return 0.86602540378443864676;
    case 2: case 10: return 0.5;
    case 3: case 9: return 0.0;
    case 4: case 8: return -0.5;
    case 5: case 7: return -0.86602540378443864676;
    default: return -1.0;
  }
}

// In-register DFT of size R1*R2 by one Cooley-Tukey split: n = R2 n1 + n2, k = k1 + R1 k2:
// DFT_R1 over n1 for each n2, twiddle exp(sign 2 pi i n2 k1 / N), DFT_R2 over n2 for each k1.
template <int R1, int R2, typename C> __device__ __forceinline__ void dft_composite(C* v, int sign) {
  using T = decltype(C::x);
  constexpr int N = R1 * R2;
  C y[R2][R1];
#pragma unroll
  for (int n2 = 0; n2 < R2; ++n2) {
    C t[R1];
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) t[n1] = v[R2 * n1 + n2];
    SmallDft<R1, C>::run(t, sign);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
      const int m = n2 * k1;
      if (m == 0) {
        y[n2][k1] = t[k1];
      } else if (N % 3 == 0 && (4 * m) % N == 0) {
        // a whole number of quarter turns: exact, by swapping and negating (N = 12 only: at
        // N = 16 the specialised code of the 128-point kernels measured slower)
        const int q = (4 * m) / N;
        const C a = t[k1];
        if (q == 2)
          y[n2][k1] = mk<C>(-a.x, -a.y);
        else if ((q == 1) == (sign > 0))
          y[n2][k1] = mk<C>(-a.y, a.x);                              // times i
        else
          y[n2][k1] = mk<C>(a.y, -a.x);                              // times -i
      } else {
        const C w = mk<C>(T(cos_frac(m, N)), T(sign) * T(cos_frac(m - N / 4, N)));
        y[n2][k1] = cmul(t[k1], w);
      }
    }
  }
#pragma unroll
  for (int k1 = 0; k1 < R1; ++k1) {
    C t[R2];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) t[n2] = y[n2][k1];
    SmallDft<R2, C>::run(t, sign);
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) v[k1 + R1 * k2] = t[k2];
  }
}

template <typename C> struct SmallDft<16, C> {
  static __device__ __forceinline__ void run(C* v, int sign) { dft_composite<4, 4, C>(v, sign); }
};
template <typename C> struct SmallDft<12, C> {
  static __device__ __forceinline__ void run(C* v, int sign) { dft_composite<4, 3, C>(v, sign); }
};

// Radix sequence: a final 12- or 16-point stage where it fits (96 = 8 x 12, 128 = 8 x 16,
// 48 = 4 x 12, 36 = 12 x 3), else 8, 4, 2, 3.
template <int N, int Ns> struct RadixOf {
  static constexpr int rem = N / Ns;
  static constexpr int R = (rem == 12 || rem == 16) ? rem
                           : (rem == 48)            ? 4
                           : (rem == 36)            ? 12
                           : (rem % 8 == 0)         ? 8
                           : (rem % 4 == 0)         ? 4
                           : (rem % 2 == 0)         ? 2
                                                    : 3;
};

// Identity epilogue of the last stage.
struct NoEpi {
  __device__ __forceinline__ float2 operator()(float2 v, int, int) const { return v; }
};

// One stage over `lines` lines (<= LPC lines; LPC = lines per call).  LINE_FAST: job =
// j * LPC + l (consecutive threads on consecutive lines), else job = l * M + j.  The last
// stage (Ns * R == N) passes every output through epi(value, element index, line index
// within the call) before storing it.
template <int N, int Ns, int R, int THREADS, int LPC, bool LINE_FAST, int SIGN, class Epi>
__device__ __forceinline__ void cstage(float2* s, int lines, int lstride, int kstride, const float2* tw,
                                       const Epi& epi) {
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
      for (int r = 0; r < R; ++r) {
        const int x = base + r * Ns;
        line[x * kstride] = (Ns * R == N) ? epi(v[q][r], x, l) : v[q][r];
      }
    }
  }
  __syncthreads();
}

template <int N, int Ns, int THREADS, int LPC, bool LINE_FAST, int SIGN, class Epi> struct CFft {
  static __device__ __forceinline__ void run(float2* s, int lines, int lstride, int kstride, const float2* tw,
                                             const Epi& epi) {
    constexpr int R = RadixOf<N, Ns>::R;
    cstage<N, Ns, R, THREADS, LPC, LINE_FAST, SIGN, Epi>(s, lines, lstride, kstride, tw, epi);
    CFft<N, Ns * R, THREADS, LPC, LINE_FAST, SIGN, Epi>::run(s, lines, lstride, kstride, tw, epi);
  }
};
template <int N, int THREADS, int LPC, bool LINE_FAST, int SIGN, class Epi>
struct CFft<N, N, THREADS, LPC, LINE_FAST, SIGN, Epi> {
  static __device__ __forceinline__ void run(float2*, int, int, int, const float2*, const Epi&) {}
};

// Shifts the line index of an epilogue by the first line of a call.
template <class Epi> struct EpiAt {
  const Epi& e;
  int l0;
  __device__ __forceinline__ float2 operator()(float2 v, int x, int l) const { return e(v, x, l0 + l); }
};

// All `lines` lines, LPC at a time; epi(value, element, line) on the last stage's outputs.
template <int N, int THREADS, int LPC, bool LINE_FAST, int SIGN, class Epi = NoEpi>
__device__ __forceinline__ void cfft_lines(float2* s, int lines, int lstride, int kstride, const float2* tw,
                                           const Epi& epi = Epi()) {
  for (int l0 = 0; l0 < lines; l0 += LPC)
    CFft<N, 1, THREADS, LPC, LINE_FAST, SIGN, EpiAt<Epi>>::run(s + l0 * lstride, min(LPC, lines - l0), lstride,
                                                                kstride, tw, EpiAt<Epi>{epi, l0});
}

}  // namespace ks
