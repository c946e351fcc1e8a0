// Full-grid ("plain") path kernels: batched line FFTs, sphere scatter/gather with the
// kinetic term, potential multiply, real-space KB projectors (Eq. 9), density (Eq. 1),
// periodic Poisson + Slater exchange, and the FP64 reductions for norms and energies.
#include <type_traits>

#include "fft_device.cuh"
#include "kernels.h"

namespace ks {

namespace {

constexpr int RED_THREADS = 256;

// Deterministic block sum of NV doubles per thread; result valid in thread 0.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
  __shared__ double red[32][NV];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i)
    for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], o);
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) red[warp][i] = v[i];
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  if (warp == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      v[i] = (lane < nw) ? red[lane][i] : 0.0;
      for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], o);
    }
  }
  __syncthreads();
}

// ------------------------------------------------------------------------------------------
// Line FFTs along one axis of [nb][N][N][N] grids.
// Lines are addressed as (outer a, inner b): element k at a*N*B + k*B + b.
// ------------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(LINE_THREADS) k_fft_lines(cplx<T>* __restrict__ data, int N, long nouter, int B,
                                                            int TB, FftPlan plan, const cplx<T>* __restrict__ twg,
                                                            int sign) {
  using C = cplx<T>;
  extern __shared__ unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* s = tw + N;
  const int ld = N + 1;
  for (int t = threadIdx.x; t < N; t += blockDim.x) {
    const C w = twg[t];
    tw[t] = mk<C>(w.x, sign > 0 ? w.y : -w.y);
  }
  int lines;
  size_t base;
  if (B == 1) {
    const long a0 = (long)blockIdx.x * TB;
    lines = (int)min((long)TB, nouter - a0);
    base = (size_t)a0 * N;
    for (int e = threadIdx.x; e < lines * N; e += blockDim.x) {
      const int l = e / N, k = e - (e / N) * N;
      s[l * ld + k] = data[base + (size_t)l * N + k];
    }
  } else {
    const int ntb = (B + TB - 1) / TB;
    const long a = blockIdx.x / ntb;
    const int b0 = (int)(blockIdx.x - a * ntb) * TB;
    lines = min(TB, B - b0);
    base = (size_t)a * N * B + b0;
    for (int e = threadIdx.x; e < lines * N; e += blockDim.x) {
      const int k = e / lines, l = e - (e / lines) * lines;
      s[l * ld + k] = data[base + (size_t)k * B + l];
    }
  }
  __syncthreads();
  fft_lines_smem(s, lines, ld, N, plan, tw, sign);
  if (B == 1) {
    for (int e = threadIdx.x; e < lines * N; e += blockDim.x) {
      const int l = e / N, k = e - (e / N) * N;
      data[base + (size_t)l * N + k] = s[l * ld + k];
    }
  } else {
    for (int e = threadIdx.x; e < lines * N; e += blockDim.x) {
      const int k = e / lines, l = e - (e / lines) * lines;
      data[base + (size_t)k * B + l] = s[l * ld + k];
    }
  }
}

template <typename T>
__global__ void k_scatter(const cplx<T>* __restrict__ psi, cplx<T>* __restrict__ grid, const int* __restrict__ gidx,
                          int nG, size_t N3) {
  const int b = blockIdx.y;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < nG; g += gridDim.x * blockDim.x)
    grid[b * N3 + gidx[g]] = psi[(size_t)b * nG + g];
}

template <typename T>
__global__ void k_gather_kinetic(const cplx<T>* __restrict__ grid, const cplx<T>* __restrict__ psi,
                                 cplx<T>* __restrict__ hpsi, const int* __restrict__ gidx, const T* __restrict__ g2h,
                                 int nG, size_t N3, T scale) {
  const int b = blockIdx.y;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < nG; g += gridDim.x * blockDim.x) {
    const cplx<T> u = grid[b * N3 + gidx[g]];
    if (psi) {
      const cplx<T> p = psi[(size_t)b * nG + g];
      const T k = g2h[g];
      hpsi[(size_t)b * nG + g] = mk<cplx<T>>(u.x * scale + k * p.x, u.y * scale + k * p.y);
    } else {
      hpsi[(size_t)b * nG + g] = mk<cplx<T>>(u.x * scale, u.y * scale);
    }
  }
}

template <typename T>
__global__ void k_multiply_potential(cplx<T>* __restrict__ grid, const T* __restrict__ v, size_t N3) {
  const int b = blockIdx.y;
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < N3; j += (size_t)gridDim.x * blockDim.x) {
    const T vj = v[j];
    cplx<T> u = grid[b * N3 + j];
    grid[b * N3 + j] = mk<cplx<T>>(u.x * vj, u.y * vj);
  }
}

// grid[j] *= exp(i kappa . (r_j - L/2)), r_j = h (jx, jy, jz), row-major z fastest
template <typename T>
__global__ void k_multiply_phase(cplx<T>* __restrict__ grid, int N, T h, T L, T kx, T ky, T kz) {
  const size_t N3 = (size_t)N * N * N;
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < N3; j += (size_t)gridDim.x * blockDim.x) {
    const int jz = (int)(j % N), jy = (int)((j / N) % N), jx = (int)(j / ((size_t)N * N));
    const T ph = kx * (h * jx - T(0.5) * L) + ky * (h * jy - T(0.5) * L) + kz * (h * jz - T(0.5) * L);
    T sn, cs;
    if constexpr (std::is_same<T, float>::value)
      sincosf(ph, &sn, &cs);
    else
      sincos(ph, &sn, &cs);
    const cplx<T> u = grid[j];
    grid[j] = mk<cplx<T>>(u.x * cs - u.y * sn, u.x * sn + u.y * cs);
  }
}

// Forces (Eq. 11).  grid[gidx[g]] = i G_alpha c_g for one state, G = g0 m, m from the grid
// index (j < N/2: j, else j - N); the grid must be zeroed before.
template <typename T>
__global__ void k_scatter_grad(const cplx<T>* __restrict__ psi, cplx<T>* __restrict__ grid, const int* __restrict__ gidx,
                               int nG, int N, T g0, int alpha) {
  const int b = blockIdx.y;
  const size_t N3 = (size_t)N * N * N;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < nG; g += gridDim.x * blockDim.x) {
    const int idx = gidx[g];
    const int j = alpha == 0 ? idx / (N * N) : (alpha == 1 ? (idx / N) % N : idx % N);
    const T G = g0 * (T)(j < N / 2 ? j : j - N);
    const cplx<T> c = psi[(size_t)b * nG + g];
    grid[b * N3 + idx] = mk<cplx<T>>(-G * c.y, G * c.x);
  }
}

// gacc[j] += sum_b occ[b] 2 Re(conj(dpsi[b][j]) psi[b][j]), states in order, summed in T (the
// precision of gacc; FP64 arithmetic would run at 1/64 of the FP32 rate on the mixed path)
template <typename T>
__global__ void k_grad_accumulate(const cplx<T>* __restrict__ dpsi, const cplx<T>* __restrict__ psi, T* __restrict__ gacc,
                                  size_t N3, int nb, const double* __restrict__ occ) {
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < N3; j += (size_t)gridDim.x * blockDim.x) {
    T acc = 0;
    for (int b = 0; b < nb; ++b) {
      const cplx<T> d = dpsi[b * N3 + j], p = psi[b * N3 + j];
      acc += (T)(2.0 * occ[b]) * (d.x * p.x + d.y * p.y);
    }
    gacc[j] += acc;
  }
}

// fnl[3 I + alpha] -= w sum_b occ[b] sum_l Re(conj(q_bIl) p_bIl), one thread per atom (states in order)
template <typename T>
__global__ void k_nl_force(const cplx<T>* __restrict__ p, const cplx<T>* __restrict__ q, int natoms, int nproj, int nb,
                           double w, const double* __restrict__ occ, double* __restrict__ fnl, int alpha) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= natoms) return;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) {
    double sb = 0.0;
    for (int l = 0; l < nproj; ++l) {
      const size_t e = ((size_t)b * natoms + I) * nproj + l;
      const cplx<T> a = p[e], c = q[e];
      sb += (double)c.x * (double)a.x + (double)c.y * (double)a.y;
    }
    s += occ[b] * sb;
  }
  fnl[3 * I + alpha] -= w * s;
}

// floc[3 I + a] = coef sum_j X_I[jx] Y_I[jy] Z_I[jz] g_a[j], one block per atom; xyz holds per
// atom the three per-axis image sums [natoms][3][N] of the separable Gaussian
template <typename T>
__global__ void k_local_force(const T* __restrict__ g, const double* __restrict__ xyz, int N, double coef,
                              double* __restrict__ partials, int zmajor) {
  const int I = blockIdx.x, sl = blockIdx.y;
  const size_t N3 = (size_t)N * N * N;
  const size_t j0 = N3 * sl / LOCAL_FORCE_SPLIT, j1 = N3 * (sl + 1) / LOCAL_FORCE_SPLIT;
  const double* X = xyz + (size_t)I * 3 * N;
  const double* Y = X + N;
  const double* Z = Y + N;
  double acc[3] = {0.0, 0.0, 0.0};
  for (size_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
    const int a0 = (int)(j % N), a1 = (int)((j / N) % N), a2 = (int)(j / ((size_t)N * N));
    const int jz = zmajor ? a2 : a0, jy = zmajor ? a0 : a1, jx = zmajor ? a1 : a2;
    const double v = X[jx] * Y[jy] * Z[jz];
    acc[0] += v * (double)g[j];
    acc[1] += v * (double)g[N3 + j];
    acc[2] += v * (double)g[2 * N3 + j];
  }
  block_sum<3>(acc);
  if (threadIdx.x == 0)
    for (int a = 0; a < 3; ++a) partials[((size_t)I * LOCAL_FORCE_SPLIT + sl) * 3 + a] = coef * acc[a];
}

__global__ void k_local_force_finish(const double* __restrict__ partials, int natoms, double* __restrict__ floc) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;                // 3 I + a
  if (e >= 3 * natoms) return;
  const int I = e / 3, a = e % 3;
  double s = 0.0;
  for (int sl = 0; sl < LOCAL_FORCE_SPLIT; ++sl) s += partials[((size_t)I * LOCAL_FORCE_SPLIT + sl) * 3 + a];
  floc[e] = s;
}

// The local potential of Gaussian atoms from their separable 27-image axis factors.
template <typename T>
__global__ void k_vloc_from_axes(const double* __restrict__ xyz, int natoms, int N, double depth, T* __restrict__ v,
                                 double* __restrict__ v64) {
  const size_t N3 = (size_t)N * N * N;
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < N3; j += (size_t)gridDim.x * blockDim.x) {
    const int jz = (int)(j % N), jy = (int)((j / N) % N), jx = (int)(j / ((size_t)N * N));
    double acc = 0.0;
    for (int I = 0; I < natoms; ++I) {
      const double* X = xyz + (size_t)I * 3 * N;
      acc += X[jx] * X[N + jy] * X[2 * N + jz];
    }
    acc *= depth;
    v[j] = (T)acc;
    if (v64) v64[j] = acc;
  }
}

// Block partials of sum_j n_j (r_j - L/2) (three components), r_j = h (jx, jy, jz)
template <typename T>
__global__ void k_dipole_partials(const T* __restrict__ n, int N, double h, double L, double* __restrict__ partials) {
  const size_t N3 = (size_t)N * N * N;
  double acc[3] = {0.0, 0.0, 0.0};
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < N3; j += (size_t)gridDim.x * blockDim.x) {
    const int jz = (int)(j % N), jy = (int)((j / N) % N), jx = (int)(j / ((size_t)N * N));
    const double nj = (double)n[j];
    acc[0] += nj * (h * jx - 0.5 * L);
    acc[1] += nj * (h * jy - 0.5 * L);
    acc[2] += nj * (h * jz - 0.5 * L);
  }
  block_sum<3>(acc);
  if (threadIdx.x == 0)
    for (int i = 0; i < 3; ++i) partials[blockIdx.x * 3 + i] = acc[i];
}

__global__ void k_dipole_finish(const double* __restrict__ partials, int nblocks, double dV, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s[3] = {0, 0, 0};
    for (int b = 0; b < nblocks; ++b)
      for (int i = 0; i < 3; ++i) s[i] += partials[b * 3 + i];
    for (int i = 0; i < 3; ++i) out[i] = dV * s[i];
  }
}

template <typename T, int NP>
__global__ void k_nl_project(const cplx<T>* __restrict__ grid, size_t N3, const int* __restrict__ sph_off,
                             const int* __restrict__ sph_idx, const T* __restrict__ beta, int natoms,
                             cplx<T>* __restrict__ proj, T scale, int zmajor_n, const int* __restrict__ zorder) {
  const int I = blockIdx.x, b = blockIdx.y;
  double acc[2 * NP];
#pragma unroll
  for (int i = 0; i < 2 * NP; ++i) acc[i] = 0.0;
  for (int q = sph_off[I] + threadIdx.x; q < sph_off[I + 1]; q += blockDim.x) {
    // on [z][x][y] grids the points go plane by plane, so that a warp reads runs of y
    const int p = zmajor_n ? zorder[q] : q;
    int idx = sph_idx[p];
    if (zmajor_n) {                                                   // (x, y, z) -> [z][x][y]
      const int n = zmajor_n, jz = idx % n, jxy = idx / n;
      idx = jz * n * n + jxy;
    }
    const cplx<T> v = grid[b * N3 + idx];
#pragma unroll
    for (int l = 0; l < NP; ++l) {
      const double w = (double)beta[(size_t)p * NP + l];
      acc[2 * l] += w * (double)v.x;
      acc[2 * l + 1] += w * (double)v.y;
    }
  }
  block_sum<2 * NP>(acc);
  if (threadIdx.x == 0)
#pragma unroll
    for (int l = 0; l < NP; ++l)
      proj[((size_t)b * natoms + I) * NP + l] = mk<cplx<T>>(T(acc[2 * l] * scale), T(acc[2 * l + 1] * scale));
}

template <typename T, int NP>
__global__ void k_nl_add(cplx<T>* __restrict__ grid, size_t N3, int ncov, const int* __restrict__ cov_idx,
                         const int* __restrict__ cov_off, const int* __restrict__ cov_ent,
                         const int* __restrict__ sph_atom, const T* __restrict__ beta, int natoms,
                         const cplx<T>* __restrict__ proj, T scale) {
  const int b = blockIdx.y;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncov; c += gridDim.x * blockDim.x) {
    T ax = 0, ay = 0;
    for (int e = cov_off[c]; e < cov_off[c + 1]; ++e) {
      const int p = cov_ent[e];
      const cplx<T>* pr = proj + ((size_t)b * natoms + sph_atom[p]) * NP;
#pragma unroll
      for (int l = 0; l < NP; ++l) {
        const T w = beta[(size_t)p * NP + l];
        ax += w * pr[l].x;
        ay += w * pr[l].y;
      }
    }
    const size_t j = b * N3 + cov_idx[c];
    cplx<T> u = grid[j];
    grid[j] = mk<cplx<T>>(u.x + scale * ax, u.y + scale * ay);
  }
}

template <typename T>
__global__ void k_density_acc(const cplx<T>* __restrict__ grid, const double* __restrict__ occ, T* __restrict__ n,
                              size_t N3, int nb, T scale, int first) {
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < N3; j += (size_t)gridDim.x * blockDim.x) {
    T acc = 0;
    for (int b = 0; b < nb; ++b) {
      const cplx<T> v = grid[b * N3 + j];
      acc += T(occ[b]) * (v.x * v.x + v.y * v.y);
    }
    n[j] = (first ? T(0) : n[j]) + scale * acc;
  }
}

template <typename T>
__global__ void k_real_to_complex(const T* __restrict__ n, cplx<T>* __restrict__ w, size_t N3) {
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < N3; j += (size_t)gridDim.x * blockDim.x)
    w[j] = mk<cplx<T>>(n[j], T(0));
}

__device__ __forceinline__ int freq_of(int j, int N) { return (2 * j < N) ? j : j - N; }

template <typename T>
__global__ void k_poisson(cplx<T>* __restrict__ w, int N, double kf2, T scale) {
  const size_t N3 = (size_t)N * N * N;
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < N3; j += (size_t)gridDim.x * blockDim.x) {
    const int jx = (int)(j / ((size_t)N * N)), jy = (int)((j / N) % N), jz = (int)(j % N);
    const int mx = freq_of(jx, N), my = freq_of(jy, N), mz = freq_of(jz, N);
    const int m2 = mx * mx + my * my + mz * mz;
    if (m2 == 0) {
      w[j] = mk<cplx<T>>(T(0), T(0));
    } else {
      const T f = T(4.0 * M_PI / (kf2 * m2)) * scale;
      const cplx<T> v = w[j];
      w[j] = mk<cplx<T>>(v.x * f, v.y * f);
    }
  }
}

template <typename T>
__global__ void k_hxc_combine(const T* __restrict__ n, const cplx<T>* __restrict__ w, const T* __restrict__ vloc,
                              T* __restrict__ vtot, double* __restrict__ partials, size_t N3) {
  double acc[3] = {0.0, 0.0, 0.0};
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < N3; j += (size_t)gridDim.x * blockDim.x) {
    const T nj = n[j];
    const T vh = w[j].x;
    const T nn = nj > T(0) ? nj : T(0);
    const T vx = -cbrt(T(3.0 / M_PI) * nn);
    vtot[j] = vloc[j] + vh + vx;
    acc[0] += (double)nj * (double)vh;
    acc[1] += (double)nj * 0.75 * (double)vx;
    acc[2] += (double)nj * (double)vx;
  }
  block_sum<3>(acc);
  if (threadIdx.x == 0)
    for (int i = 0; i < 3; ++i) partials[blockIdx.x * 3 + i] = acc[i];
}

__global__ void k_hxc_finish(const double* __restrict__ partials, int nblocks, double dV, double* __restrict__ parts) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s[3] = {0, 0, 0};
    for (int b = 0; b < nblocks; ++b)
      for (int i = 0; i < 3; ++i) s[i] += partials[b * 3 + i];
    parts[0] = 0.5 * dV * s[0];
    parts[1] = dV * s[1];
    parts[2] = dV * s[2];
  }
}

// Linear density mixing (Sec. Ground-state solution): nin <- nin + mix (nout - nin); the
// block partials of sum |nout - nin| (before the update) give the self-consistency residual.
template <typename T>
__global__ void k_density_mix(const T* __restrict__ nout, T* __restrict__ nin, size_t N3, T mix,
                              double* __restrict__ partials) {
  double acc[1] = {0.0};
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < N3; j += (size_t)gridDim.x * blockDim.x) {
    const T a = nin[j], b = nout[j];
    acc[0] += fabs((double)b - (double)a);
    nin[j] = a + mix * (b - a);
  }
  block_sum<1>(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc[0];
}

// Pulay mixing, store step: R = nout - nin into hr, nin into hn (the history slot), and the
// block partials of sum |R|, sum R^2 and sum R r_q for the other history residuals r_q.
template <typename T>
__global__ void k_pulay_store(const T* __restrict__ nout, const T* __restrict__ nin, T* __restrict__ hn,
                              T* __restrict__ hr, size_t N3, PulayRefs<T> refs, double* __restrict__ partials) {
  double acc[2 + PULAY_MAX];
#pragma unroll
  for (int i = 0; i < 2 + PULAY_MAX; ++i) acc[i] = 0.0;
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < N3; j += (size_t)gridDim.x * blockDim.x) {
    const T a = nin[j];
    const T rr = nout[j] - a;
    hn[j] = a;
    hr[j] = rr;
    const double rd = (double)rr;
    acc[0] += fabs(rd);
    acc[1] += rd * rd;
#pragma unroll
    for (int q = 0; q < PULAY_MAX; ++q)
      if (q < refs.m) acc[2 + q] += rd * (double)refs.r[q][j];
  }
  block_sum<2 + PULAY_MAX>(acc);
  if (threadIdx.x == 0)
    for (int i = 0; i < 2 + PULAY_MAX; ++i) partials[blockIdx.x * (2 + PULAY_MAX) + i] = acc[i];
}

__global__ void k_pulay_finish(const double* __restrict__ partials, int nblocks, double dV, double* __restrict__ out) {
  const int i = threadIdx.x;
  if (blockIdx.x == 0 && i < 2 + PULAY_MAX) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += partials[b * (2 + PULAY_MAX) + i];
    out[i] = dV * s;
  }
}

// nin = sum_i a_i (n_i + mix r_i) over the history pairs
template <typename T>
__global__ void k_pulay_mix(T* __restrict__ nin, size_t N3, PulayMix<T> p) {
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < N3; j += (size_t)gridDim.x * blockDim.x) {
    double v = 0.0;
#pragma unroll
    for (int q = 0; q < PULAY_MAX; ++q)
      if (q < p.m) v += p.a[q] * (double)p.n[q][j] + p.b[q] * (double)p.r[q][j];
    nin[j] = (T)v;
  }
}

// Teter-preconditioned SD, step 1 (one block per state): tr[b] = sum_g g2half |R|^2 and
// r2[b] = sum_g |R|^2 of the residual R = hpsi - eig[b] psi.
template <typename T>
__global__ void k_residual_kinetic(const cplx<T>* __restrict__ psi, const cplx<T>* __restrict__ hpsi,
                                   const T* __restrict__ g2h, const double* __restrict__ eig, int nG,
                                   double2* __restrict__ out) {
  const int b = blockIdx.x;
  const double e = eig[b];
  double acc[2] = {0.0, 0.0};
  for (int g = threadIdx.x; g < nG; g += blockDim.x) {
    const cplx<T> p = psi[(size_t)b * nG + g], h = hpsi[(size_t)b * nG + g];
    const double rx = (double)h.x - e * (double)p.x, ry = (double)h.y - e * (double)p.y;
    const double r2 = rx * rx + ry * ry;
    acc[0] += (double)g2h[g] * r2;
    acc[1] += r2;
  }
  block_sum<2>(acc);
  if (threadIdx.x == 0) out[b] = make_double2(acc[0], acc[1]);
}

// Step 2: psi -= alpha_b K(g2half / T_b) R with T_b = max(tr / r2, tmin), alpha_b = 1 / (T_b + shift);
// K(x) = (27 + 18x + 12x^2 + 8x^3) / (27 + 18x + 12x^2 + 8x^3 + 16x^4).  States with R = 0 stay.
template <typename T>
__global__ void k_teter_update(cplx<T>* __restrict__ psi, const cplx<T>* __restrict__ hpsi, const T* __restrict__ g2h,
                               const double* __restrict__ eig, const double2* __restrict__ trr, double shift,
                               double tmin, int nG) {
  const int b = blockIdx.y;
  const double2 q = trr[b];
  if (!(q.y > 0.0)) return;                                          // uniform per block
  const double t = fmax(q.x / q.y, tmin);
  const T inv_t = (T)(1.0 / t), alpha = (T)(1.0 / (t + shift)), e = (T)eig[b];
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < nG; g += gridDim.x * blockDim.x) {
    const T x = g2h[g] * inv_t;
    const T p = T(27) + x * (T(18) + x * (T(12) + x * T(8)));
    const T k = alpha * p / (p + T(16) * x * x * x * x);
    cplx<T> c = psi[(size_t)b * nG + g];
    const cplx<T> h = hpsi[(size_t)b * nG + g];
    c.x -= k * (h.x - e * c.x);
    c.y -= k * (h.y - e * c.y);
    psi[(size_t)b * nG + g] = c;
  }
}

__global__ void k_sum_partials(const double* __restrict__ partials, int nblocks, double scale, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += partials[b];
    *out = scale * s;
  }
}

template <typename T>
__global__ void k_state_dots(const cplx<T>* __restrict__ a, const cplx<T>* __restrict__ bb, int nG,
                             double2* __restrict__ dots) {
  const int b = blockIdx.x;
  double acc[2] = {0.0, 0.0};
  if constexpr (std::is_same<T, float>::value) {
    // complex64 states: FP32 products summed in FP32 over runs of 8 of a thread's elements, the
    // runs summed in FP64 (FP64 arithmetic runs at 1/64 of the FP32 rate: per element it took
    // 3 ms per 512-state td128 block; each run carries at most 16 FP32 roundings)
    float p0 = 0.f, p1 = 0.f;
    int k = 0;
    for (int g = threadIdx.x; g < nG; g += blockDim.x) {
      const cplx<T> x = a[(size_t)b * nG + g], y = bb[(size_t)b * nG + g];
      p0 = fmaf(x.x, y.x, p0);
      p0 = fmaf(x.y, y.y, p0);
      p1 = fmaf(x.x, y.y, p1);
      p1 = fmaf(-x.y, y.x, p1);
      if (++k == 8) {
        acc[0] += (double)p0;
        acc[1] += (double)p1;
        p0 = p1 = 0.f;
        k = 0;
      }
    }
    acc[0] += (double)p0;
    acc[1] += (double)p1;
  } else {
    for (int g = threadIdx.x; g < nG; g += blockDim.x) {
      const cplx<T> x = a[(size_t)b * nG + g], y = bb[(size_t)b * nG + g];
      acc[0] += (double)x.x * y.x + (double)x.y * y.y;
      acc[1] += (double)x.x * y.y - (double)x.y * y.x;
    }
  }
  block_sum<2>(acc);
  if (threadIdx.x == 0) dots[b] = make_double2(acc[0], acc[1]);
}

__global__ void k_weighted_energy(const double2* __restrict__ dots, const double* __restrict__ occ, int nb,
                                  const double* __restrict__ parts, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double e = 0;
    for (int b = 0; b < nb; ++b) e += occ[b] * dots[b].x;
    if (parts) e += -parts[0] + parts[1] - parts[2];
    out[0] = e;
  }
}

template <typename T>
__global__ void k_axpy2(cplx<T>* __restrict__ acc1, double2 a1, cplx<T>* __restrict__ acc2, double2 a2,
                        const cplx<T>* __restrict__ w, const cplx<T>* __restrict__ base, size_t n) {
  const T a1x = T(a1.x), a1y = T(a1.y), a2x = T(a2.x), a2y = T(a2.y);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const cplx<T> v = w[i];
    const cplx<T> b = base ? base[i] : acc1[i];
    cplx<T> p = b;
    p.x += a1x * v.x - a1y * v.y;
    p.y += a1x * v.y + a1y * v.x;
    acc1[i] = p;
    if (acc2) {
      cplx<T> q = base ? b : acc2[i];
      q.x += a2x * v.x - a2y * v.y;
      q.y += a2x * v.y + a2y * v.x;
      acc2[i] = q;
    }
  }
}

// SplitMix64 (Steele, Lea, Flood 2014), used as a counter-based hash.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

template <typename T>
__global__ void k_random_states(cplx<T>* __restrict__ psi, size_t n, uint64_t seed) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const uint64_t a = splitmix64(seed ^ (2 * i)), b = splitmix64(seed ^ (2 * i + 1));
    const double u = (double)(a >> 11) * (1.0 / 9007199254740992.0) - 0.5;
    const double v = (double)(b >> 11) * (1.0 / 9007199254740992.0) - 0.5;
    psi[i] = mk<cplx<T>>(T(u), T(v));
  }
}

template <typename T>
__global__ void k_from_c128(const double2* __restrict__ in, cplx<T>* __restrict__ out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = mk<cplx<T>>(T(in[i].x), T(in[i].y));
}
template <typename T>
__global__ void k_to_c128(const cplx<T>* __restrict__ in, double2* __restrict__ out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = make_double2((double)in[i].x, (double)in[i].y);
}
template <typename T>
__global__ void k_real_to_double(const T* __restrict__ in, double* __restrict__ out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = (double)in[i];
}

inline unsigned blocks_for(size_t n, int threads, unsigned cap = 152u * 16u) {
  size_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  return (unsigned)(b < cap ? b : cap);
}

}  // namespace

// ------------------------------------------------------------------------------------------
// Launchers
// ------------------------------------------------------------------------------------------
template <typename T>
void fft_axis(cplx<T>* grid, int nb, int N, int axis, int sign, const cplx<T>* tw, cudaStream_t s) {
  const FftPlan plan = make_plan(N);
  long nouter;
  int B;
  if (axis == 2) {
    nouter = (long)nb * N * N;
    B = 1;
  } else if (axis == 1) {
    nouter = (long)nb * N;
    B = N;
  } else {
    nouter = nb;
    B = N * N;
  }
  int TB = LINE_ELEMS / N;
  if (B > 1 && TB > B) TB = B;
  long nblocks = (B == 1) ? (nouter + TB - 1) / TB : nouter * ((B + TB - 1) / TB);
  const size_t smem = (size_t)(N + TB * (N + 1)) * sizeof(cplx<T>);
  k_fft_lines<T><<<(unsigned)nblocks, LINE_THREADS, smem, s>>>(grid, N, nouter, B, TB, plan, tw, sign);
  KS_CHECK_LAUNCH();
}

template <typename T>
void scatter_sphere(const cplx<T>* psi, cplx<T>* grid, const DevTables<T>& t, int nb, cudaStream_t s) {
  dim3 g(blocks_for(t.nG, 256, 1024), nb);
  k_scatter<T><<<g, 256, 0, s>>>(psi, grid, t.gidx, t.nG, (size_t)t.N * t.N * t.N);
  KS_CHECK_LAUNCH();
}

template <typename T>
void gather_kinetic(const cplx<T>* grid, const cplx<T>* psi, cplx<T>* hpsi, const DevTables<T>& t, int nb, T scale,
                    cudaStream_t s) {
  dim3 g(blocks_for(t.nG, 256, 1024), nb);
  k_gather_kinetic<T><<<g, 256, 0, s>>>(grid, psi, hpsi, t.gidx, t.g2half, t.nG, (size_t)t.N * t.N * t.N, scale);
  KS_CHECK_LAUNCH();
}

template <typename T>
void multiply_potential(cplx<T>* grid, const T* v, int N3, int nb, cudaStream_t s) {
  dim3 g(blocks_for(N3, 256, 2048), nb);
  k_multiply_potential<T><<<g, 256, 0, s>>>(grid, v, (size_t)N3);
  KS_CHECK_LAUNCH();
}

template <typename T>
void multiply_phase(cplx<T>* grid, int N, double L, const double kappa[3], cudaStream_t s) {
  const size_t N3 = (size_t)N * N * N;
  k_multiply_phase<T><<<blocks_for(N3, 256, 2048), 256, 0, s>>>(grid, N, (T)(L / N), (T)L, (T)kappa[0], (T)kappa[1],
                                                                 (T)kappa[2]);
  KS_CHECK_LAUNCH();
}

template <typename T>
void scatter_grad(const cplx<T>* psi, cplx<T>* grid, const DevTables<T>& t, int alpha, int nb, cudaStream_t s) {
  k_scatter_grad<T><<<dim3(blocks_for((size_t)t.nG, 256, 1024), nb), 256, 0, s>>>(psi, grid, t.gidx, t.nG, t.N,
                                                                                   (T)(2.0 * M_PI / t.L), alpha);
  KS_CHECK_LAUNCH();
}

template <typename T>
void grad_accumulate(const cplx<T>* dpsi, const cplx<T>* psi, T* gacc, int N3, int nb, const double* occ,
                     cudaStream_t s) {
  k_grad_accumulate<T><<<blocks_for((size_t)N3, 256, 2048), 256, 0, s>>>(dpsi, psi, gacc, (size_t)N3, nb, occ);
  KS_CHECK_LAUNCH();
}

template <typename T>
void nl_force(const cplx<T>* p, const cplx<T>* q, int natoms, int nproj, int nb, double w, const double* occ,
              double* fnl, int alpha, cudaStream_t s) {
  k_nl_force<T><<<(natoms + 127) / 128, 128, 0, s>>>(p, q, natoms, nproj, nb, w, occ, fnl, alpha);
  KS_CHECK_LAUNCH();
}

template <typename T>
void local_force(const T* g, const double* xyz, int N, int natoms, double coef, double* partials, double* floc,
                 cudaStream_t s, bool zmajor) {
  k_local_force<T><<<dim3(natoms, LOCAL_FORCE_SPLIT), RED_THREADS, 0, s>>>(g, xyz, N, coef, partials, zmajor ? 1 : 0);
  KS_CHECK_LAUNCH();
  k_local_force_finish<<<(3 * natoms + 127) / 128, 128, 0, s>>>(partials, natoms, floc);
  KS_CHECK_LAUNCH();
}

template <typename T>
__global__ void k_grad_packed(const cplx<T>* __restrict__ psi, cplx<T>* __restrict__ out, const int* __restrict__ gidx,
                              int nG, int N, T g0, int alpha) {
  const int b = blockIdx.y;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < nG; g += gridDim.x * blockDim.x) {
    const int idx = gidx[g];
    const int j = alpha == 0 ? idx / (N * N) : (alpha == 1 ? (idx / N) % N : idx % N);
    const T G = g0 * (T)(j < N / 2 ? j : j - N);
    const cplx<T> c = psi[(size_t)b * nG + g];
    out[(size_t)b * nG + g] = mk<cplx<T>>(-G * c.y, G * c.x);
  }
}

template <typename T>
void grad_packed(const cplx<T>* psi, cplx<T>* out, const DevTables<T>& t, int alpha, int nb, cudaStream_t s) {
  k_grad_packed<T><<<dim3(blocks_for((size_t)t.nG, 256, 1024), nb), 256, 0, s>>>(psi, out, t.gidx, t.nG, t.N,
                                                                                  (T)(2.0 * M_PI / t.L), alpha);
  KS_CHECK_LAUNCH();
}

template <typename T>
void vloc_from_axes(const double* xyz, int natoms, int N, double depth, T* v, double* v64, cudaStream_t s) {
  const size_t N3 = (size_t)N * N * N;
  k_vloc_from_axes<T><<<blocks_for(N3, 256, 4096), 256, 0, s>>>(xyz, natoms, N, depth, v, v64);
  KS_CHECK_LAUNCH();
}

template <typename T>
void dipole(const T* n, int N, double L, double* partials, int nblocks, double* out, cudaStream_t s) {
  k_dipole_partials<T><<<nblocks, RED_THREADS, 0, s>>>(n, N, L / N, L, partials);
  KS_CHECK_LAUNCH();
  k_dipole_finish<<<1, 32, 0, s>>>(partials, nblocks, (L / N) * (L / N) * (L / N), out);
  KS_CHECK_LAUNCH();
}

template <typename T>
void nl_project(const cplx<T>* grid, const DevTables<T>& t, cplx<T>* proj, int nb, T scale, cudaStream_t s,
                bool zmajor) {
  if (t.natoms == 0) return;
  dim3 g(t.natoms, nb);
  const size_t N3 = (size_t)t.N * t.N * t.N;
  const int zn = zmajor ? t.N : 0;
  if (t.nproj == 4)
    k_nl_project<T, 4><<<g, RED_THREADS, 0, s>>>(grid, N3, t.sph_off, t.sph_idx, t.sph_beta, t.natoms, proj, scale, zn,
                                                 t.sph_zorder);
  else
    k_nl_project<T, 1><<<g, RED_THREADS, 0, s>>>(grid, N3, t.sph_off, t.sph_idx, t.sph_beta, t.natoms, proj, scale, zn,
                                                 t.sph_zorder);
  KS_CHECK_LAUNCH();
}

template <typename T>
void nl_add(cplx<T>* grid, const DevTables<T>& t, const cplx<T>* proj, int nb, T scale, cudaStream_t s) {
  if (t.natoms == 0 || t.ncov == 0) return;
  dim3 g(blocks_for(t.ncov, 256, 1024), nb);
  const size_t N3 = (size_t)t.N * t.N * t.N;
  if (t.nproj == 4)
    k_nl_add<T, 4><<<g, 256, 0, s>>>(grid, N3, t.ncov, t.cov_idx, t.cov_off, t.cov_ent, t.sph_atom, t.sph_beta,
                                     t.natoms, proj, scale);
  else
    k_nl_add<T, 1><<<g, 256, 0, s>>>(grid, N3, t.ncov, t.cov_idx, t.cov_off, t.cov_ent, t.sph_atom, t.sph_beta,
                                     t.natoms, proj, scale);
  KS_CHECK_LAUNCH();
}

template <typename T>
void density_accumulate(const cplx<T>* grid, const double* occ, T* n, int N3, int nb, T scale, bool first,
                        cudaStream_t s) {
  k_density_acc<T><<<blocks_for(N3, 256, 4096), 256, 0, s>>>(grid, occ, n, (size_t)N3, nb, scale, first ? 1 : 0);
  KS_CHECK_LAUNCH();
}

template <typename T>
void real_to_complex(const T* n, cplx<T>* work, int N3, cudaStream_t s) {
  k_real_to_complex<T><<<blocks_for(N3, 256, 4096), 256, 0, s>>>(n, work, (size_t)N3);
  KS_CHECK_LAUNCH();
}

template <typename T>
void poisson_multiply(cplx<T>* work, int N, double L, T scale, cudaStream_t s) {
  const double kf = 2.0 * M_PI / L;
  k_poisson<T><<<blocks_for((size_t)N * N * N, 256, 4096), 256, 0, s>>>(work, N, kf * kf, scale);
  KS_CHECK_LAUNCH();
}

template <typename T>
void hxc_combine(const T* n, const cplx<T>* work, const T* vloc, T* vtot, double* partials, int N3, int nblocks,
                 cudaStream_t s) {
  k_hxc_combine<T><<<nblocks, RED_THREADS, 0, s>>>(n, work, vloc, vtot, partials, (size_t)N3);
  KS_CHECK_LAUNCH();
}

void hxc_finish(const double* partials, int nblocks, double dV, double* parts, cudaStream_t s) {
  k_hxc_finish<<<1, 32, 0, s>>>(partials, nblocks, dV, parts);
  KS_CHECK_LAUNCH();
}

template <typename T>
void density_mix(const T* nout, T* nin, int N3, double mix, double* partials, int nblocks, cudaStream_t s) {
  k_density_mix<T><<<nblocks, RED_THREADS, 0, s>>>(nout, nin, (size_t)N3, (T)mix, partials);
  KS_CHECK_LAUNCH();
}

template <typename T>
void pulay_store(const T* nout, const T* nin, T* hn, T* hr, int N3, const PulayRefs<T>& refs, double* partials,
                 int nblocks, double dV, double* out, cudaStream_t s) {
  k_pulay_store<T><<<nblocks, RED_THREADS, 0, s>>>(nout, nin, hn, hr, (size_t)N3, refs, partials);
  KS_CHECK_LAUNCH();
  k_pulay_finish<<<1, 32, 0, s>>>(partials, nblocks, dV, out);
  KS_CHECK_LAUNCH();
}

template <typename T>
void pulay_mix(T* nin, int N3, const PulayMix<T>& p, cudaStream_t s) {
  k_pulay_mix<T><<<blocks_for((size_t)N3, 256, 2048), 256, 0, s>>>(nin, (size_t)N3, p);
  KS_CHECK_LAUNCH();
}

template <typename T>
void teter_update(cplx<T>* psi, const cplx<T>* hpsi, const T* g2half, const double* eig, double2* trr, double shift,
                  double tmin, int nG, int n, cudaStream_t s) {
  k_residual_kinetic<T><<<n, RED_THREADS, 0, s>>>(psi, hpsi, g2half, eig, nG, trr);
  KS_CHECK_LAUNCH();
  k_teter_update<T><<<dim3(blocks_for((size_t)nG, 256, 64), n), 256, 0, s>>>(psi, hpsi, g2half, eig, trr, shift,
                                                                            tmin, nG);
  KS_CHECK_LAUNCH();
}

__global__ void k_minmax_partials(const double* __restrict__ v, size_t n, double* __restrict__ partials) {
  __shared__ double smin[RED_THREADS], smax[RED_THREADS];
  double lo = INFINITY, hi = -INFINITY;
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < n; j += (size_t)gridDim.x * blockDim.x) {
    lo = fmin(lo, v[j]);
    hi = fmax(hi, v[j]);
  }
  smin[threadIdx.x] = lo;
  smax[threadIdx.x] = hi;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w /= 2) {
    if ((int)threadIdx.x < w) {
      smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + w]);
      smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = smin[0];
    partials[2 * blockIdx.x + 1] = smax[0];
  }
}

__global__ void k_minmax_finish(const double* __restrict__ partials, int nblocks, double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double lo = INFINITY, hi = -INFINITY;
  for (int b = 0; b < nblocks; ++b) {
    lo = fmin(lo, partials[2 * b]);
    hi = fmax(hi, partials[2 * b + 1]);
  }
  out[0] = lo;
  out[1] = hi;
}

void minmax(const double* v, size_t n, double* partials, int nblocks, double* out, cudaStream_t s) {
  k_minmax_partials<<<nblocks, RED_THREADS, 0, s>>>(v, n, partials);
  KS_CHECK_LAUNCH();
  k_minmax_finish<<<1, 32, 0, s>>>(partials, nblocks, out);
  KS_CHECK_LAUNCH();
}

void sum_partials(const double* partials, int nblocks, double scale, double* out, cudaStream_t s) {
  k_sum_partials<<<1, 32, 0, s>>>(partials, nblocks, scale, out);
  KS_CHECK_LAUNCH();
}

template <typename T>
void state_dots(const cplx<T>* a, const cplx<T>* b, int nG, int nb, double2* dots, cudaStream_t s) {
  k_state_dots<T><<<nb, RED_THREADS, 0, s>>>(a, b, nG, dots);
  KS_CHECK_LAUNCH();
}

void weighted_energy(const double2* dots, const double* occ, int nb, const double* parts, double* out, cudaStream_t s) {
  k_weighted_energy<<<1, 32, 0, s>>>(dots, occ, nb, parts, out);
  KS_CHECK_LAUNCH();
}

template <typename T>
void axpy2(cplx<T>* acc1, double2 a1, cplx<T>* acc2, double2 a2, const cplx<T>* w, const cplx<T>* base, size_t n,
           cudaStream_t s) {
  k_axpy2<T><<<blocks_for(n, 256, 152 * 32), 256, 0, s>>>(acc1, a1, acc2, a2, w, base, n);
  KS_CHECK_LAUNCH();
}


template <typename T>
void random_states(cplx<T>* psi, size_t n, uint64_t seed, cudaStream_t s) {
  k_random_states<T><<<blocks_for(n, 256), 256, 0, s>>>(psi, n, seed);
  KS_CHECK_LAUNCH();
}

template <typename T>
void from_c128(const double2* in, cplx<T>* out, size_t n, cudaStream_t s) {
  k_from_c128<T><<<blocks_for(n, 256), 256, 0, s>>>(in, out, n);
  KS_CHECK_LAUNCH();
}
template <typename T>
void to_c128(const cplx<T>* in, double2* out, size_t n, cudaStream_t s) {
  k_to_c128<T><<<blocks_for(n, 256), 256, 0, s>>>(in, out, n);
  KS_CHECK_LAUNCH();
}
template <typename T>
void real_to_double(const T* in, double* out, size_t n, cudaStream_t s) {
  k_real_to_double<T><<<blocks_for(n, 256), 256, 0, s>>>(in, out, n);
  KS_CHECK_LAUNCH();
}

#define KS_INSTANTIATE(T)                                                                                       \
  template void fft_axis<T>(cplx<T>*, int, int, int, int, const cplx<T>*, cudaStream_t);                        \
  template void scatter_sphere<T>(const cplx<T>*, cplx<T>*, const DevTables<T>&, int, cudaStream_t);            \
  template void gather_kinetic<T>(const cplx<T>*, const cplx<T>*, cplx<T>*, const DevTables<T>&, int, T,        \
                                  cudaStream_t);                                                                \
  template void multiply_potential<T>(cplx<T>*, const T*, int, int, cudaStream_t);                              \
  template void nl_project<T>(const cplx<T>*, const DevTables<T>&, cplx<T>*, int, T, cudaStream_t, bool);       \
  template void nl_add<T>(cplx<T>*, const DevTables<T>&, const cplx<T>*, int, T, cudaStream_t);                 \
  template void density_accumulate<T>(const cplx<T>*, const double*, T*, int, int, T, bool, cudaStream_t);      \
  template void real_to_complex<T>(const T*, cplx<T>*, int, cudaStream_t);                                      \
  template void poisson_multiply<T>(cplx<T>*, int, double, T, cudaStream_t);                                    \
  template void hxc_combine<T>(const T*, const cplx<T>*, const T*, T*, double*, int, int, cudaStream_t);        \
  template void density_mix<T>(const T*, T*, int, double, double*, int, cudaStream_t);                          \
  template void pulay_store<T>(const T*, const T*, T*, T*, int, const PulayRefs<T>&, double*, int, double, double*, \
                               cudaStream_t);                                                                   \
  template void pulay_mix<T>(T*, int, const PulayMix<T>&, cudaStream_t);                                        \
  template void teter_update<T>(cplx<T>*, const cplx<T>*, const T*, const double*, double2*, double, double, int, \
                                int,                                                                            \
                                cudaStream_t);                                                                  \
  template void multiply_phase<T>(cplx<T>*, int, double, const double*, cudaStream_t);                          \
  template void dipole<T>(const T*, int, double, double*, int, double*, cudaStream_t);                          \
  template void scatter_grad<T>(const cplx<T>*, cplx<T>*, const DevTables<T>&, int, int, cudaStream_t);         \
  template void grad_accumulate<T>(const cplx<T>*, const cplx<T>*, T*, int, int, const double*, cudaStream_t);  \
  template void nl_force<T>(const cplx<T>*, const cplx<T>*, int, int, int, double, const double*, double*, int,  \
                            cudaStream_t);                                                                      \
  template void local_force<T>(const T*, const double*, int, int, double, double*, double*, cudaStream_t, bool); \
  template void grad_packed<T>(const cplx<T>*, cplx<T>*, const DevTables<T>&, int, int, cudaStream_t);          \
  template void vloc_from_axes<T>(const double*, int, int, double, T*, double*, cudaStream_t);                  \
  template void state_dots<T>(const cplx<T>*, const cplx<T>*, int, int, double2*, cudaStream_t);                \
  template void axpy2<T>(cplx<T>*, double2, cplx<T>*, double2, const cplx<T>*, const cplx<T>*, size_t, cudaStream_t);           \
  template void random_states<T>(cplx<T>*, size_t, uint64_t, cudaStream_t);                                     \
  template void from_c128<T>(const double2*, cplx<T>*, size_t, cudaStream_t);                                   \
  template void to_c128<T>(const cplx<T>*, double2*, size_t, cudaStream_t);                                     \
  template void real_to_double<T>(const T*, double*, size_t, cudaStream_t);

KS_INSTANTIATE(float)
KS_INSTANTIATE(double)

}  // namespace ks
