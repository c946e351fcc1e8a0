// Fused mixed-precision H psi (complex64), three kernels per application:
//
//   k_zinv   packed sphere coefficients -> inverse z-FFT of the sphere's z-columns only
//            -> column buffer [state][z][column]
//   k_plane  one (state, z-plane) per CTA, the N x N plane in shared memory: scatter the
//            columns, inverse y-FFT on the rows that hold columns, inverse x-FFT on every
//            line, u = V psi + sum_{I,l} D beta_Il p_Il (projector add on the sphere points
//            of this plane), forward x-FFT, forward y-FFT on the rows that hold columns,
//            gather the columns -> second column buffer
//   k_zfwd   forward z-FFT of the columns, keep G in S, scale N^-3, add |G|^2/2 c
//
// The projections p_Il = dV sum_j beta_Il(r_j) psi(r_j) (Eq. 9) are computed before the
// plane pass, in Fourier space: on the grid, by Parseval, p_Il = sum_{G in S}
// conj(b_Il(G)) c_G with b_Il the sphere coefficients of the grid function beta_Il (built
// at setup, and again when the atoms move, by a separable FP64 DFT over each atom's box).
// That is one overlap GEMM of the projector block with
// the state block; the add stays in real space, fused into the plane kernel.
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>

#include "fft_device.cuh"
#include "fused.h"

namespace ks {

namespace {


struct PlaneNL {
  const int* pt_off;     // [N+1] covered points of plane z
  const int* pt_xy;      // jx*N + jy
  const int* ent_off;    // [npts+1]
  const int* ent_proj;   // first projector row (atom * nproj)
  const float* ent_beta; // [nent][nproj]
  int nproj;
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((unsigned)__cvta_generic_to_shared(smem)), "l"(gmem));
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((unsigned)__cvta_generic_to_shared(smem)), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Per-size launch shapes: plane kernel threads (and CTAs per SM), lines per FFT call
// (at most 8 complex values per thread per stage), z-kernel columns per CTA.
template <int N> struct FCfg {
  static constexpr int PT = N >= 128 ? 1024 : (N >= 64 ? 512 : 256);
  static constexpr int PMIN = N >= 128 ? 1 : (N >= 64 ? 2 : 4);
  // lines per call: at most 8 complex per thread per stage; 96 takes 32 so that three calls
  // cover the 96 x-lines exactly and no warp straddles two lines' radix jobs
  static constexpr int LPC = N == 96 ? 32 : ((8 * PT / N) < N ? (8 * PT / N) : N);
  static constexpr int ZT = 512;
  static constexpr int CT = (4096 / N) < 32 ? (4096 / N) : 32;
};

// Column c of the sphere holds 2h+1 consecutive coefficients (h = col_half[c]) starting at
// col_off[c], z-indices 0..h then N-h..N-1: coefficient k has z = k for k <= h, else
// k + N - 2h - 1.  The z-kernels derive a coefficient's (column, z) from these two numbers.
// k_zinv takes ZSB consecutive states per CTA for one block of CT columns and keeps two
// column blocks in shared memory: while one state's block is transformed, the next state's
// coefficients arrive by asynchronous copies (software pipelining hides the load latency that
// one block per CTA left exposed).  Dynamic shared memory: twiddles [N], then the two blocks
// [CT][N + 1].
constexpr int ZSB = 4;
template <int N> constexpr size_t zsmem() { return (size_t)(N + 2 * FCfg<N>::CT * (N + 1)) * sizeof(float2); }

template <int N>
__global__ void __launch_bounds__(FCfg<N>::ZT, 2) k_zinv(const float2* __restrict__ psi, int nG, const int* __restrict__ col_off,
                                                      const int* __restrict__ col_half, int ncols, int nstates,
                                                      float2* __restrict__ colbuf, const float2* __restrict__ twg) {
  constexpr int CT = FCfg<N>::CT, ld = N + 1, ZT = FCfg<N>::ZT;
  extern __shared__ __align__(16) float2 zsm[];
  float2* tw = zsm;
  float2* sb[2] = {zsm + N, zsm + N + CT * ld};
  __shared__ int coff[CT], chalf[CT];
  const int b0 = blockIdx.y * ZSB;
  const int nb = min(ZSB, nstates - b0);
  const int c0 = blockIdx.x * CT;
  const int nl = min(CT, ncols - c0);
  for (int t = threadIdx.x; t < N; t += ZT) tw[t] = twg[t];
  for (int t = threadIdx.x; t < nl; t += ZT) {
    coff[t] = col_off[c0 + t];
    chalf[t] = col_half[c0 + t];
  }
  __syncthreads();
  // slot z of column l holds coefficient k = z (z <= h) or z - (N - 2h - 1) (z >= N - h); the
  // other slots are zero in both blocks (set here, and again after each block is stored)
  constexpr int TPC = ZT / CT, SLOTS = (N + TPC - 1) / TPC;
  const int l = threadIdx.x / TPC, sub = threadIdx.x - (threadIdx.x / TPC) * TPC;
  const int h = l < nl ? chalf[l] : -1, g0 = l < nl ? coff[l] : 0;
  if (l < nl) {
#pragma unroll
    for (int q = 0; q < SLOTS; ++q) {
      const int z = sub + q * TPC;
      if (z < N && z > h && z < N - h) {
        sb[0][l * ld + z] = make_float2(0.f, 0.f);
        sb[1][l * ld + z] = make_float2(0.f, 0.f);
      }
    }
  }
  auto issue = [&](int i) {                                          // state b0 + i -> block i & 1
    if (l >= nl) return;
    const float2* col = psi + (size_t)(b0 + i) * nG + g0;
    float2* dst = sb[i & 1] + l * ld;
#pragma unroll
    for (int q = 0; q < SLOTS; ++q) {
      const int z = sub + q * TPC;
      if (z < N) {
        const int k = z <= h ? z : (z >= N - h ? z - (N - 2 * h - 1) : -1);
        if (k >= 0) cp_async8(dst + z, col + k);
      }
    }
  };
  issue(0);
  cp_async_commit();
  for (int i = 0; i < nb; ++i) {
    if (i + 1 < nb) {
      issue(i + 1);
      cp_async_commit();
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    } else {
      cp_async_wait_all();
    }
    __syncthreads();
    float2* s = sb[i & 1];
    cfft_lines<N, ZT, CT, true, +1>(s, nl, ld, 1, tw);
    // transpose out: element e = z * CT + lc; slots outside the column's range go back to zero
    float2* out = colbuf + (size_t)(b0 + i) * N * ncols + c0;
#pragma unroll
    for (int q = 0; q < (N * CT + ZT - 1) / ZT; ++q) {
      const int e = threadIdx.x + q * ZT;
      const int z = e / CT, lc = e % CT;
      if (z < N && lc < nl) {
        out[(size_t)z * ncols + lc] = s[lc * ld + z];
        const int hc = chalf[lc];
        if (z > hc && z < N - hc) s[lc * ld + z] = make_float2(0.f, 0.f);
      }
    }
    __syncthreads();                                                  // block i & 1 free for state i + 2
  }
}

// k_zfwd: one state per CTA (blockIdx.y); the column block arrives by asynchronous copies
// while the state's psi and |G|^2/2 load into registers.  (A ZSB-state pipelined form like
// k_zinv's spilled: the next block's copy addresses and the write-back indices stayed live
// across the transform.)
template <int N>
__global__ void __launch_bounds__(FCfg<N>::ZT, 3) k_zfwd(const float2* __restrict__ colbuf, const float2* __restrict__ psi,
                                                      float2* __restrict__ hpsi, int nG, const int* __restrict__ col_off,
                                                      const int* __restrict__ col_half, const float* __restrict__ g2half,
                                                      int ncols, float scale, const float2* __restrict__ twg) {
  constexpr int CT = FCfg<N>::CT, ld = N + 1, ZT = FCfg<N>::ZT;
  __shared__ float2 tw[N];
  __shared__ float2 s[CT * ld];
  __shared__ int coff[CT], chalf[CT];
  const int b = blockIdx.y;
  const int c0 = blockIdx.x * CT;
  const int nl = min(CT, ncols - c0);
  for (int t = threadIdx.x; t < N; t += ZT) tw[t] = twg[t];
  for (int t = threadIdx.x; t < nl; t += ZT) {
    coff[t] = col_off[c0 + t];
    chalf[t] = col_half[c0 + t];
  }
  __syncthreads();
  // the coefficients this thread finally writes: psi and |G|^2/2 are loaded now, so that their
  // latency hides behind the column loads and the FFT (a group of TPC threads per column)
  constexpr int TPC = ZT / CT, GS = (N + TPC - 1) / TPC, LOADS = (N * CT + ZT - 1) / ZT;
  const size_t off = (size_t)b * nG;
  const int l = threadIdx.x / TPC, sub = threadIdx.x - (threadIdx.x / TPC) * TPC;
  const int h = l < nl ? chalf[l] : -1, g0 = l < nl ? coff[l] : 0;
  float2 pv[GS];
  float kv[GS];
#pragma unroll
  for (int q = 0; q < GS; ++q) {
    const int k = sub + q * TPC;
    if (k <= 2 * h) {
      pv[q] = psi[off + g0 + k];
      kv[q] = g2half[g0 + k];
    }
  }
  // the column block, transposed into the line layout by 8-byte asynchronous copies
  const float2* in = colbuf + (size_t)b * N * ncols + c0;
#pragma unroll
  for (int q = 0; q < LOADS; ++q) {
    const int e = threadIdx.x + q * ZT;
    const int z = e / CT, lc = e % CT;
    if (z < N && lc < nl) cp_async8(&s[lc * ld + z], &in[(size_t)z * ncols + lc]);
  }
  cp_async_commit();
  cp_async_wait_all();
  __syncthreads();
  cfft_lines<N, ZT, CT, true, -1>(s, nl, ld, 1, tw);
#pragma unroll
  for (int q = 0; q < GS; ++q) {
    const int k = sub + q * TPC;
    if (k <= 2 * h) {
      const int z = k <= h ? k : k + N - 2 * h - 1;
      const float2 u = s[l * ld + z];
      hpsi[off + g0 + k] = make_float2(u.x * scale + kv[q] * pv[q].x, u.y * scale + kv[q] * pv[q].y);
    }
  }
}

// Zero the plane, scatter the columns of one (state, z-plane), inverse y transforms of the
// rows that hold columns.  The first column loads are issued before the plane is cleared, so
// their latency overlaps it.
template <int N>
__device__ __forceinline__ void plane_load_y(float2* P, const float2* __restrict__ colrow, int ncols,
                                             const int* __restrict__ col_xy, int xr, const float2* tw) {
  constexpr int ld = N + 1, PT = FCfg<N>::PT, LPC = FCfg<N>::LPC, EARLY = 4;
  float2 cv[EARLY];
  int cxy[EARLY];
#pragma unroll
  for (int e = 0; e < EARLY; ++e) {
    const int c = threadIdx.x + e * PT;
    if (c < ncols) {
      cv[e] = colrow[c];
      cxy[e] = col_xy[c];
    }
  }
  for (int e = threadIdx.x; e < N * ld; e += PT) P[e] = make_float2(0.f, 0.f);
  __syncthreads();
#pragma unroll
  for (int e = 0; e < EARLY; ++e) {
    const int c = threadIdx.x + e * PT;
    if (c < ncols) {
      const int jx = cxy[e] / N, jy = cxy[e] - (cxy[e] / N) * N;
      P[jx * ld + jy] = cv[e];
    }
  }
  for (int c = threadIdx.x + EARLY * PT; c < ncols; c += PT) {
    const int xy = col_xy[c];
    const int jx = xy / N, jy = xy - jx * N;
    P[jx * ld + jy] = colrow[c];
  }
  __syncthreads();
  // y-lines of the rows that hold columns: jx in [0, xr] and [N - xr, N - 1].  Every line pass
  // puts consecutive threads on consecutive lines: with the odd row pitch N + 1 a warp's
  // 8-byte accesses then fall on distinct bank pairs.
  cfft_lines<N, PT, LPC, true, +1>(P, xr + 1, ld, 1, tw);
  if (xr > 0) cfft_lines<N, PT, LPC, true, +1>(P + (N - xr) * ld, xr, ld, 1, tw);
}

// u = V psi as the last stage of the inverse x transform stores it (x = jx, line = jy).
template <int N> struct VMul {
  const float* V;
  __device__ __forceinline__ float2 operator()(float2 v, int x, int l) const {
    const float vv = V[x * N + l];
    return make_float2(v.x * vv, v.y * vv);
  }
};

// Dynamic shared memory: twiddles [N], plane [N][N+1], V plane [N*N] (float), then this
// state's projections [nprojtot] when pf_smem.  V and the projections are fetched with
// cp.async at entry and land while the inverse transforms run.
template <int N>
__global__ void __launch_bounds__(FCfg<N>::PT, FCfg<N>::PMIN)
    k_plane(const float2* __restrict__ colbuf1, float2* __restrict__ colbuf2, int ncols, const int* __restrict__ col_xy,
            int xr, const float* __restrict__ vplane, PlaneNL nl, const float2* __restrict__ pf, int nprojtot,
            int pf_smem, const float2* __restrict__ twg) {
  constexpr int ld = N + 1, PT = FCfg<N>::PT, LPC = FCfg<N>::LPC;
  extern __shared__ __align__(16) float2 psm[];
  float2* tw = psm;
  float2* P = psm + N;
  float* Vs = reinterpret_cast<float*>(P + N * ld);
  float2* pfs = reinterpret_cast<float2*>(Vs + N * N);
  const int z = blockIdx.x, b = blockIdx.y;
  const float* vsrc = vplane + (size_t)z * N * N;
  for (int c = threadIdx.x; c < N * N / 4; c += PT) cp_async16(Vs + 4 * c, vsrc + 4 * c);
  if (pf_smem)
    for (int q = threadIdx.x; q < nprojtot; q += PT) cp_async8(pfs + q, pf + (size_t)b * nprojtot + q);
  cp_async_commit();
  int pt0 = 0, pt1 = 0;
  if (nprojtot > 0) {
    pt0 = nl.pt_off[z];
    pt1 = nl.pt_off[z + 1];
  }
  for (int t = threadIdx.x; t < N; t += PT) tw[t] = twg[t];
  const size_t row = ((size_t)b * N + z) * ncols;
  plane_load_y<N>(P, colbuf1 + row, ncols, col_xy, xr, tw);
  cp_async_wait_all();
  __syncthreads();
  // inverse x transforms; the last stage stores u = V psi
  cfft_lines<N, PT, LPC, true, +1>(P, N, 1, ld, tw, VMul<N>{Vs});
  // + sum_{I,l} D Omega^{1/2} beta_Il p_Il  (pf already carries D Omega^{1/2})
  if (nprojtot > 0) {
    const float2* pb = pf_smem ? pfs : pf + (size_t)b * nprojtot;
    for (int pt = pt0 + threadIdx.x; pt < pt1; pt += PT) {
      const int xy = nl.pt_xy[pt];
      const int e0 = nl.ent_off[pt], e1 = nl.ent_off[pt + 1];
      float ax = 0.f, ay = 0.f;
      for (int e = e0; e < e1; ++e) {
        const float2* pp = pb + nl.ent_proj[e];
        const float* bt = nl.ent_beta + (size_t)e * nl.nproj;
        for (int l = 0; l < nl.nproj; ++l) {
          ax += bt[l] * pp[l].x;
          ay += bt[l] * pp[l].y;
        }
      }
      const int jx = xy / N, jy = xy - jx * N;
      const float2 u = P[jx * ld + jy];
      P[jx * ld + jy] = make_float2(u.x + ax, u.y + ay);
    }
  }
  __syncthreads();
  // forward x-lines (all), then y-lines of the rows that hold columns
  cfft_lines<N, PT, LPC, true, -1>(P, N, 1, ld, tw);
  cfft_lines<N, PT, LPC, true, -1>(P, xr + 1, ld, 1, tw);
  if (xr > 0) cfft_lines<N, PT, LPC, true, -1>(P + (N - xr) * ld, xr, ld, 1, tw);
  for (int c = threadIdx.x; c < ncols; c += PT) {
    const int xy = col_xy[c];
    const int jx = xy / N, jy = xy - jx * N;
    colbuf2[row + c] = P[jx * ld + jy];
  }
}

// Real-space planes of the states (forces, Eq. 11, need psi and its gradient on the grid):
// one (state, z-plane) per CTA, the inverse y and x passes of k_plane, then the plane is
// stored contiguously at out[b][z] ([x][y], row pitch N).
template <int N>
__global__ void __launch_bounds__(FCfg<N>::PT, FCfg<N>::PMIN)
    k_plane_inverse(const float2* __restrict__ colbuf1, int ncols, const int* __restrict__ col_xy, int xr,
                    const float2* __restrict__ twg, float2* __restrict__ out) {
  constexpr int ld = N + 1, PT = FCfg<N>::PT, LPC = FCfg<N>::LPC;
  extern __shared__ __align__(16) float2 psm[];
  float2* tw = psm;
  float2* P = psm + N;
  const int z = blockIdx.x, b = blockIdx.y;
  for (int t = threadIdx.x; t < N; t += PT) tw[t] = twg[t];
  const size_t row = ((size_t)b * N + z) * ncols;
  plane_load_y<N>(P, colbuf1 + row, ncols, col_xy, xr, tw);
  cfft_lines<N, PT, LPC, true, +1>(P, N, 1, ld, tw);
  float2* o = out + ((size_t)b * N + z) * N * N;
  for (int e = threadIdx.x; e < N * N; e += PT) o[e] = P[(e / N) * ld + (e - (e / N) * N)];
}

// Density partial sums: one (z-plane, state) per CTA; a cluster holds DCL consecutive states
// of one plane.  Each CTA transforms its state and writes f |u|^2 into its own shared-memory
// plane (fused into the last stage of the inverse x transform).  The cluster then sums its
// DCL planes through distributed shared memory, rank by rank in a fixed order, each CTA a
// slice of the plane.  One state per CTA keeps the transforms free of a loop over states,
// which would hold their index arithmetic live and spill.
constexpr int DCL = 8;

template <int N> struct DensSet {
  float* acc;
  float f;
  __device__ __forceinline__ float2 operator()(float2 v, int x, int l) const {
    acc[x * N + l] = f * (v.x * v.x + v.y * v.y);
    return v;
  }
};

template <int N>
__global__ void __cluster_dims__(1, DCL, 1) __launch_bounds__(FCfg<N>::PT, FCfg<N>::PMIN)
    k_plane_density(const float2* __restrict__ colbuf1, int ncols, const int* __restrict__ col_xy, int xr,
                    int nstates, const double* __restrict__ occ, float scale, float* __restrict__ partial,
                    const float2* __restrict__ twg) {
  namespace cg = cooperative_groups;
  constexpr int ld = N + 1, PT = FCfg<N>::PT, LPC = FCfg<N>::LPC;
  extern __shared__ __align__(16) float2 psm[];
  float2* tw = psm;
  float2* P = psm + N;
  float* acc = reinterpret_cast<float*>(P + N * ld);
  const int z = blockIdx.x, b = blockIdx.y;
  for (int t = threadIdx.x; t < N; t += PT) tw[t] = twg[t];
  if (b < nstates) {
    // the y transforms (their first barrier also publishes tw), then the x transforms
    plane_load_y<N>(P, colbuf1 + ((size_t)b * N + z) * ncols, ncols, col_xy, xr, tw);
    cfft_lines<N, PT, LPC, true, +1>(P, N, 1, ld, tw, DensSet<N>{acc, (float)occ[b]});
  } else {
    for (int e = threadIdx.x; e < N * N; e += PT) acc[e] = 0.f;   // padding state of the cluster
  }
  cg::cluster_group cl = cg::this_cluster();
  cl.sync();
  const int r = (int)cl.block_rank();
  constexpr int E = (N * N + DCL - 1) / DCL;
  float* out = partial + ((size_t)(b / DCL) * N + z) * N * N;
  const int e1 = min(N * N, (r + 1) * E);
  for (int e = r * E + threadIdx.x; e < e1; e += PT) {
    float sum = 0.f;
#pragma unroll
    for (int q = 0; q < DCL; ++q) sum += cl.map_shared_rank(acc, q)[e];
    out[e] = sum * scale;
  }
  cl.sync();                                                         // keep the planes until read
}

// The same partial sums with one (z-plane, chunk of states) per CTA, states in order, for
// the grids whose plane CTA fills an SM alone (N = 128: 1024 threads), where a cluster's
// synchronisation and reduction per state would be exposed.  f |u|^2 is accumulated in the
// last stage of the inverse x transform (each point by one thread, in state order).
template <int N> struct DensAcc {
  float* acc;
  float f;
  __device__ __forceinline__ float2 operator()(float2 v, int x, int l) const {
    acc[x * N + l] += f * (v.x * v.x + v.y * v.y);
    return v;
  }
};

template <int N>
__global__ void __launch_bounds__(FCfg<N>::PT, FCfg<N>::PMIN)
    k_plane_density_chunk(const float2* __restrict__ colbuf1, int ncols, const int* __restrict__ col_xy, int xr,
                          int nstates, int chunk, const double* __restrict__ occ, float scale,
                          float* __restrict__ partial, const float2* __restrict__ twg) {
  constexpr int ld = N + 1, PT = FCfg<N>::PT, LPC = FCfg<N>::LPC;
  extern __shared__ __align__(16) float2 psm[];
  float2* tw = psm;
  float2* P = psm + N;
  float* acc = reinterpret_cast<float*>(P + N * ld);
  const int z = blockIdx.x, ch = blockIdx.y;
  for (int t = threadIdx.x; t < N; t += PT) tw[t] = twg[t];
  for (int e = threadIdx.x; e < N * N; e += PT) acc[e] = 0.f;
  const int b0 = ch * chunk, b1 = min(nstates, b0 + chunk);
#pragma unroll 1
  for (int b = b0; b < b1; ++b) {
    plane_load_y<N>(P, colbuf1 + ((size_t)b * N + z) * ncols, ncols, col_xy, xr, tw);
    cfft_lines<N, PT, LPC, true, +1>(P, N, 1, ld, tw, DensAcc<N>{acc, (float)occ[b]});
  }
  float* out = partial + ((size_t)ch * N + z) * N * N;
  for (int e = threadIdx.x; e < N * N; e += PT) out[e] = acc[e] * scale;
}

// n[(jx*N + jy)*N + z] = sum_ch partial[ch][z][jx*N + jy]
__global__ void k_density_reduce(const float* __restrict__ partial, int nch, int N, float* __restrict__ n) {
  const size_t N3 = (size_t)N * N * N;
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < N3; j += (size_t)gridDim.x * blockDim.x) {
    const int z = (int)(j % N);
    const size_t xy = j / N;
    float s = 0.f;
    for (int ch = 0; ch < nch; ++ch) s += partial[((size_t)ch * N + z) * N * N + xy];
    n[j] = s;
  }
}

// vplane[z][jx*N + jy] = v[(jx*N + jy)*N + z]
__global__ void k_to_planes(const float* __restrict__ v, int N, float* __restrict__ vplane) {
  const size_t N3 = (size_t)N * N * N;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < N3; e += (size_t)gridDim.x * blockDim.x) {
    const size_t z = e / ((size_t)N * N), xy = e % ((size_t)N * N);
    vplane[e] = v[xy * N + z];
  }
}

// pf[b][ip] = scale * (float) pout[ip][b]
__global__ void k_proj_to_states(const double2* __restrict__ pout, int nprojtot, int nst, float scale,
                                 float2* __restrict__ pf) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nprojtot * nst; e += gridDim.x * blockDim.x) {
    const int b = e / nprojtot, ip = e - b * nprojtot;
    const double2 v = pout[(size_t)ip * nst + b];
    pf[e] = make_float2((float)(v.x * scale), (float)(v.y * scale));
  }
}

// Setup: projector grid functions -> sphere coefficients (FP64), then rounded to complex64.
// The projector block by a separable DFT over each atom's box of grid points (Sec.
// "Pseudopotentials": beta_Il lives on the sphere |r - R_I| < R_c, so its sphere coefficients
// are a DFT of a function supported on a small box).  Box coordinates b = 0..B-1 stand for the
// unwrapped grid index lo + b of the atom's minimum-image sphere; exp(-2 pi i m j / N) is
// periodic in j, so the unwrapped index gives the phase directly.  FP32, like the block it
// fills (the sums run over at most B ~ 2 R_c / h + 2 terms per axis).
//   T1[p][bx][by][mz] = sum_bz beta[p][bx][by][bz] e(mz (lo_z + bz))
//   T2[p][bx][my][mz] = sum_by T1[p][bx][by][mz] e(my (lo_y + by))
//   B[p][G]          = scale sum_bx T2[p][bx][my][mz] e(mx (lo_x + bx)),  e(t) = exp(-2 pi i t / N)
// with m_y, m_z in [-xr, xr] stored at index m + xr.
__device__ __forceinline__ int mod_n(long v, int N) {
  const int r = (int)(v % N);
  return r < 0 ? r + N : r;
}

__global__ void k_box_dft_z(const float* __restrict__ box, const int* __restrict__ lo, int nproj, int nrows, int B,
                            int xr, int N, const float2* __restrict__ tw, float2* __restrict__ T1) {
  const int M = 2 * xr + 1;
  const size_t total = (size_t)nrows * B * B * M;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int mi = (int)(e % M);
    const size_t pb = e / M;                                          // (p, bx, by)
    const int p = (int)(pb / ((size_t)B * B));
    const int m = mi - xr;
    const int step = mod_n(m, N);
    int t = mod_n((long)m * lo[3 * (p / nproj) + 2], N);
    const float* v = box + pb * B;
    float ax = 0.f, ay = 0.f;
    for (int bz = 0; bz < B; ++bz) {
      const float2 w = tw[t];                                         // (cos, sin)(2 pi t / N)
      ax += v[bz] * w.x;
      ay -= v[bz] * w.y;
      t += step;
      if (t >= N) t -= N;
    }
    T1[e] = make_float2(ax, ay);
  }
}

__global__ void k_box_dft_y(const float2* __restrict__ T1, const int* __restrict__ lo, int nproj, int nrows, int B,
                            int xr, int N, const float2* __restrict__ tw, float2* __restrict__ T2) {
  const int M = 2 * xr + 1;
  const size_t total = (size_t)nrows * B * M * M;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int mz = (int)(e % M);
    const int my = (int)((e / M) % M);
    const size_t pbx = e / ((size_t)M * M);                           // (p, bx)
    const int p = (int)(pbx / B);
    const int m = my - xr;
    const int step = mod_n(m, N);
    int t = mod_n((long)m * lo[3 * (p / nproj) + 1], N);
    const float2* v = T1 + pbx * B * M + mz;                         // v[by * M]
    float ax = 0.f, ay = 0.f;
    for (int by = 0; by < B; ++by) {
      const float2 w = tw[t], x = v[(size_t)by * M];
      ax += x.x * w.x + x.y * w.y;                                    // x * conj(w)
      ay += x.y * w.x - x.x * w.y;
      t += step;
      if (t >= N) t -= N;
    }
    T2[e] = make_float2(ax, ay);
  }
}

__global__ void k_box_dft_x(const float2* __restrict__ T2, const int* __restrict__ lo, const int* __restrict__ gidx,
                            int nproj, int nrows, int B, int xr, int N, int nG, float scale,
                            const float2* __restrict__ tw, float2* __restrict__ out) {
  const int M = 2 * xr + 1;
  const size_t total = (size_t)nrows * nG;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int g = (int)(e % nG);
    const int p = (int)(e / nG);
    const int idx = gidx[g];
    const int jx = idx / (N * N), jy = (idx / N) % N, jz = idx % N;
    const int mx = 2 * jx < N ? jx : jx - N, my = 2 * jy < N ? jy : jy - N, mz = 2 * jz < N ? jz : jz - N;
    const int step = mod_n(mx, N);
    int t = mod_n((long)mx * lo[3 * (p / nproj)], N);
    const float2* v = T2 + (size_t)p * B * M * M + (size_t)(my + xr) * M + (mz + xr);   // v[bx * M * M]
    float ax = 0.f, ay = 0.f;
    for (int bx = 0; bx < B; ++bx) {
      const float2 w = tw[t], x = v[(size_t)bx * M * M];
      ax += x.x * w.x + x.y * w.y;
      ay += x.y * w.x - x.x * w.y;
      t += step;
      if (t >= N) t -= N;
    }
    out[e] = make_float2(ax * scale, ay * scale);
  }
}

unsigned nblk(size_t n, int t, unsigned cap = 4096) {
  size_t b = (n + t - 1) / t;
  return (unsigned)std::max<size_t>(1, std::min<size_t>(b, cap));
}

class FusedImpl final : public FusedOps {
 public:
  static bool supported(int N) {
    switch (N) {
      case 18: case 24: case 32: case 36: case 48: case 64: case 96: case 128: return true;
      default: return false;
    }
  }

  FusedImpl(const HostGeometry& g, const DevTables<float>& t, int nstates, DeviceArena& arena, StageProfiler& prof,
            int* err)
      : g_(g), t_(t), ns_(nstates), arena_(arena), prof_(prof), err_(err) {
    N_ = g.N;
    ncols_ = g.ncols;
    nprojtot_ = g.natoms * g.nproj;
    const size_t N3 = (size_t)N_ * N_ * N_;
    build_plane_lists();
    // buffers
    colbuf1_ = alloc<float2>((size_t)ns_ * N_ * ncols_);
    colbuf2_ = alloc<float2>((size_t)ns_ * N_ * ncols_);
    vplane_ = alloc<float>(N3);
    if (nprojtot_ > 0) {
      B_ = alloc<float2>((size_t)nprojtot_ * g.nG);
      Bimg_ = arena_.alloc(tc_overlap_image_bytes(nprojtot_, g.nG));
      pout_ = alloc<double2>((size_t)nprojtot_ * ns_);
      pf_ = alloc<float2>((size_t)nprojtot_ * ns_);
      part_elems_ = std::max<size_t>(tc_overlap_part_elems(nprojtot_, ns_, true), 4096);
      part_ = alloc<double2>(part_elems_);
      build_projector_block();
    }
    nch_max_ = (ns_ + density_chunk() - 1) / density_chunk();
    dpartial_ = alloc<float>((size_t)nch_max_ * N3);
  }

  void apply_h(const float2* psi, float2* hpsi, int n, const float* v, cudaStream_t s) override {
    const size_t N3 = (size_t)N_ * N_ * N_;
    k_to_planes<<<nblk(N3, 256), 256, 0, s>>>(v, N_, vplane_);
    KS_CHECK_LAUNCH();
    if (nprojtot_ > 0) {
      ProfScope ps(prof_, "proj_gemm", s);
      tc_overlap(B_, g_.nG, psi, g_.nG, nprojtot_, n, g_.nG, part_, part_elems_, pout_, err_, s, nullptr, Bimg_);
      const float scale = (float)(g_.D * std::sqrt(g_.omega));
      k_proj_to_states<<<nblk((size_t)nprojtot_ * n, 256), 256, 0, s>>>(pout_, nprojtot_, n, scale, pf_);
      KS_CHECK_LAUNCH();
    }
    zinv(psi, n, s);
    {
      ProfScope ps(prof_, "plane", s);
      dispatch([&](auto tag) { launch_plane<decltype(tag)::value>(n, s); });
    }
    {
      ProfScope ps(prof_, "zfwd", s);
      dispatch([&](auto tag) { launch_zfwd<decltype(tag)::value>(psi, hpsi, n, s); });
    }
  }

  void real_space(const float2* psi, int n, float2* out, cudaStream_t s) override {
    zinv(psi, n, s);
    ProfScope ps(prof_, "plane_inverse", s);
    dispatch([&](auto tag) { launch_plane_inverse<decltype(tag)::value>(n, out, s); });
  }

  void prepare_atoms() override {
    plane_lists_host();
    lists_ready_ = true;
  }

  void set_atoms(const DevTables<float>& t) override {
    if (!lists_ready_) plane_lists_host();
    lists_ready_ = false;
    KS_CUDA(cudaDeviceSynchronize());
    t_ = t;
    arena_.release(nl_.pt_off);
    arena_.release(nl_.pt_xy);
    arena_.release(nl_.ent_off);
    arena_.release(nl_.ent_proj);
    arena_.release(nl_.ent_beta);
    upload_plane_lists();
    if (nprojtot_ > 0) build_projector_block();
  }

  void density(const float2* psi, int n, const double* occ, float* nout, cudaStream_t s) override {
    zinv(psi, n, s);
    ProfScope ps(prof_, "plane_density", s);
    const int nch = (n + density_chunk() - 1) / density_chunk();
    dispatch([&](auto tag) { launch_density<decltype(tag)::value>(n, nch, occ, s); });
    k_density_reduce<<<nblk((size_t)N_ * N_ * N_, 256), 256, 0, s>>>(dpartial_, nch, N_, nout);
    KS_CHECK_LAUNCH();
  }

 private:
  template <int V> struct IntTag {
    static constexpr int value = V;
  };
  template <typename F> void dispatch(F&& f) {
    switch (N_) {
      case 18: f(IntTag<18>{}); break;
      case 24: f(IntTag<24>{}); break;
      case 32: f(IntTag<32>{}); break;
      case 36: f(IntTag<36>{}); break;
      case 48: f(IntTag<48>{}); break;
      case 64: f(IntTag<64>{}); break;
      case 96: f(IntTag<96>{}); break;
      case 128: f(IntTag<128>{}); break;
      default: fail(KS_ERR_ARG, "fused path: unsupported grid %d", N_);
    }
  }

  void zinv(const float2* psi, int n, cudaStream_t s) {
    ProfScope ps(prof_, "zinv", s);
    dispatch([&](auto tag) { launch_zinv<decltype(tag)::value>(psi, n, s); });
  }

  template <int N> void launch_zinv(const float2* psi, int n, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
      KS_CUDA(cudaFuncSetAttribute(k_zinv<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zsmem<N>()));
      attr = true;
    }
    dim3 grid((ncols_ + FCfg<N>::CT - 1) / FCfg<N>::CT, (n + ZSB - 1) / ZSB);
    k_zinv<N><<<grid, FCfg<N>::ZT, zsmem<N>(), s>>>(psi, g_.nG, t_.col_off, t_.col_half, ncols_, n, colbuf1_, t_.tw);
    KS_CHECK_LAUNCH();
  }
  template <int N> void launch_zfwd(const float2* psi, float2* hpsi, int n, cudaStream_t s) {
    dim3 grid((ncols_ + FCfg<N>::CT - 1) / FCfg<N>::CT, n);
    k_zfwd<N><<<grid, FCfg<N>::ZT, 0, s>>>(colbuf2_, psi, hpsi, g_.nG, t_.col_off, t_.col_half, t_.g2half, ncols_,
                                           (float)(1.0 / ((double)N * N * N)), t_.tw);
    KS_CHECK_LAUNCH();
  }
  template <int N> static size_t plane_smem() { return (size_t)(N + N * (N + 1)) * sizeof(float2); }
  static constexpr size_t SMEM_MAX = 227 * 1024;
  template <int N> void launch_plane(int n, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
      KS_CUDA(cudaFuncSetAttribute(k_plane<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_MAX));
      attr = true;
    }
    const size_t base = plane_smem<N>() + (size_t)N * N * sizeof(float);
    const size_t with_pf = base + (size_t)nprojtot_ * sizeof(float2);
    const int pf_smem = with_pf <= SMEM_MAX;
    if (base > SMEM_MAX) fail(KS_ERR_ARG, "plane kernel: %zu bytes of shared memory for N=%d", base, N);
    dim3 grid(N, n);
    k_plane<N><<<grid, FCfg<N>::PT, pf_smem ? with_pf : base, s>>>(colbuf1_, colbuf2_, ncols_, t_.col_xy, g_.xr,
                                                                   vplane_, nl_, pf_, nprojtot_, pf_smem, t_.tw);
    KS_CHECK_LAUNCH();
  }
  template <int N> void launch_plane_inverse(int n, float2* out, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
      KS_CUDA(cudaFuncSetAttribute(k_plane_inverse<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_MAX));
      attr = true;
    }
    k_plane_inverse<N><<<dim3(N, n), FCfg<N>::PT, plane_smem<N>(), s>>>(colbuf1_, ncols_, t_.col_xy, g_.xr, t_.tw,
                                                                         out);
    KS_CHECK_LAUNCH();
  }
  // states per density partial: a cluster of DCL states, or a chunk per CTA at N = 128
  int density_chunk() const { return N_ >= 128 ? std::max(1, std::min(32, (ns_ + 7) / 8)) : DCL; }

  template <int N> void launch_density(int n, int nch, const double* occ, cudaStream_t s) {
    const size_t smem = plane_smem<N>() + (size_t)N * N * sizeof(float);
    if constexpr (N >= 128) {
      static bool attr = false;
      if (!attr) {
        KS_CUDA(cudaFuncSetAttribute(k_plane_density_chunk<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)SMEM_MAX));
        attr = true;
      }
      k_plane_density_chunk<N><<<dim3(N, nch), FCfg<N>::PT, smem, s>>>(
          colbuf1_, ncols_, t_.col_xy, g_.xr, n, density_chunk(), occ, (float)(1.0 / g_.omega), dpartial_, t_.tw);
    } else {
      static bool attr = false;
      if (!attr) {
        KS_CUDA(cudaFuncSetAttribute(k_plane_density<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_MAX));
        attr = true;
      }
      k_plane_density<N><<<dim3(N, nch * DCL), FCfg<N>::PT, smem, s>>>(   // whole clusters of DCL states
          colbuf1_, ncols_, t_.col_xy, g_.xr, n, occ, (float)(1.0 / g_.omega), dpartial_, t_.tw);
    }
    KS_CHECK_LAUNCH();
  }

  // Per-plane projector lists from the geometry's inverse lists: the covered points of each
  // z-plane, each with its sphere entries (first projector row and the nproj beta values).
  void build_plane_lists() {
    plane_lists_host();
    upload_plane_lists();
  }
  void plane_lists_host() {
    const HostGeometry& g = g_;
    std::vector<int>& pt_off = h_pt_off_;
    std::vector<int>& pt_xy = h_pt_xy_;
    std::vector<int>& ent_off = h_ent_off_;
    std::vector<int>& ent_proj = h_ent_proj_;
    std::vector<float>& ent_beta = h_ent_beta_;
    pt_off.assign(N_ + 1, 0);
    pt_xy.clear();
    ent_off.assign(1, 0);
    ent_proj.clear();
    ent_beta.clear();
    std::vector<std::vector<int>> byz(N_);
    for (size_t c = 0; c < g.cov_idx.size(); ++c) byz[g.cov_idx[c] % N_].push_back((int)c);
    for (int z = 0; z < N_; ++z) {
      for (int c : byz[z]) {
        pt_xy.push_back(g.cov_idx[c] / N_);
        for (int e = g.cov_off[c]; e < g.cov_off[c + 1]; ++e) {
          const int p = g.cov_ent[e];
          ent_proj.push_back(g.sph_atom[p] * g.nproj);
          for (int l = 0; l < g.nproj; ++l) ent_beta.push_back((float)g.sph_beta[(size_t)p * g.nproj + l]);
        }
        ent_off.push_back((int)ent_proj.size());
      }
      pt_off[z + 1] = (int)pt_xy.size();
    }
  }
  void upload_plane_lists() {
    nl_.pt_off = upload(h_pt_off_);
    nl_.pt_xy = upload(h_pt_xy_);
    nl_.ent_off = upload(h_ent_off_);
    nl_.ent_proj = upload(h_ent_proj_);
    nl_.ent_beta = upload(h_ent_beta_);
    nl_.nproj = g_.nproj;
  }

  // B[atom*nproj + l][G] = c_G[beta_Il] = Omega^{1/2} N^-3 sum_j exp(-iG.r_j) beta_Il(r_j), by the
  // separable DFT over each atom's box (k_box_dft_*), FP32.
  void build_projector_block() {
    const HostGeometry& g = g_;
    const int N = N_, na = g.natoms, np = g.nproj;
    int xr = 0;                                                       // max |m| over S, every axis
    for (int v : g.mvec) xr = std::max(xr, std::abs(v));
    const int M = 2 * xr + 1;
    // unwrapped grid coordinates of the sphere points (the minimum image of build_atoms) and
    // the box that holds each atom's sphere
    std::vector<int> lo(3 * (size_t)na, 0), hi(3 * (size_t)na, 0), ju(3 * g.sph_idx.size());
    int B = 1;
    for (int a = 0; a < na; ++a) {
      for (int p = g.sph_off[a]; p < g.sph_off[a + 1]; ++p) {
        const int idx = g.sph_idx[p];
        const int j3[3] = {idx / (N * N), (idx / N) % N, idx % N};
        for (int k = 0; k < 3; ++k) {
          const double t = j3[k] * g.h - g.pos[3 * a + k];
          const int u = j3[k] - N * (int)std::nearbyint(t / g.L);
          ju[3 * (size_t)p + k] = u;
          if (p == g.sph_off[a] || u < lo[3 * a + k]) lo[3 * a + k] = u;
          if (p == g.sph_off[a] || u > hi[3 * a + k]) hi[3 * a + k] = u;
        }
      }
      if (g.sph_off[a + 1] > g.sph_off[a])
        for (int k = 0; k < 3; ++k) B = std::max(B, hi[3 * a + k] - lo[3 * a + k] + 1);
    }
    std::vector<float> box((size_t)nprojtot_ * B * B * B, 0.f);
    for (int a = 0; a < na; ++a)
      for (int p = g.sph_off[a]; p < g.sph_off[a + 1]; ++p) {
        const size_t bx = ju[3 * (size_t)p] - lo[3 * a], by = ju[3 * (size_t)p + 1] - lo[3 * a + 1],
                     bz = ju[3 * (size_t)p + 2] - lo[3 * a + 2];
        for (int l = 0; l < np; ++l)
          box[(((size_t)(a * np + l) * B + bx) * B + by) * B + bz] = (float)g.sph_beta[(size_t)p * np + l];
      }
    // rows in chunks of whole atoms (the intermediate sums of a chunk stay below ~64 MB)
    const size_t per_row = (size_t)B * M * (B + M) * sizeof(float2);
    const int chunk = np * std::max(1, (int)std::min<size_t>(na, (size_t(64) << 20) / (per_row * np)));
    float* dbox = nullptr;
    int* dlo = nullptr;
    float2 *T1 = nullptr, *T2 = nullptr;
    const float2* tw = t_.tw;                                         // (cos, sin)(2 pi t / N), FP32
    KS_CUDA(cudaMalloc(&dbox, box.size() * sizeof(float)));
    KS_CUDA(cudaMalloc(&dlo, std::max<size_t>(1, lo.size()) * sizeof(int)));
    KS_CUDA(cudaMalloc(&T1, (size_t)chunk * B * B * M * sizeof(float2)));
    KS_CUDA(cudaMalloc(&T2, (size_t)chunk * B * M * M * sizeof(float2)));
    KS_CUDA(cudaMemcpy(dbox, box.data(), box.size() * sizeof(float), cudaMemcpyHostToDevice));
    KS_CUDA(cudaMemcpy(dlo, lo.data(), lo.size() * sizeof(int), cudaMemcpyHostToDevice));
    const float scale = (float)(std::sqrt(g.omega) / ((double)N * N * N));
    for (int r0 = 0; r0 < nprojtot_; r0 += chunk) {                   // r0: a multiple of np
      const int nr = std::min(chunk, nprojtot_ - r0);
      const int* clo = dlo + 3 * (r0 / np);
      k_box_dft_z<<<nblk((size_t)nr * B * B * M, 256), 256>>>(dbox + (size_t)r0 * B * B * B, clo, np, nr, B, xr, N,
                                                               tw, T1);
      KS_CHECK_LAUNCH();
      k_box_dft_y<<<nblk((size_t)nr * B * M * M, 256), 256>>>(T1, clo, np, nr, B, xr, N, tw, T2);
      KS_CHECK_LAUNCH();
      k_box_dft_x<<<nblk((size_t)nr * g.nG, 256), 256>>>(T2, clo, t_.gidx, np, nr, B, xr, N, g.nG, scale, tw,
                                                         B_ + (size_t)r0 * g.nG);
      KS_CHECK_LAUNCH();
    }
    tc_overlap_prepare_a(B_, g.nG, nprojtot_, g.nG, Bimg_, nullptr);   // the operand split once
    KS_CUDA(cudaStreamSynchronize(nullptr));
    cudaFree(dbox);
    cudaFree(dlo);
    cudaFree(T1);
    cudaFree(T2);
  }

  template <typename U> U* alloc(size_t n) { return static_cast<U*>(arena_.alloc(n * sizeof(U))); }
  template <typename U> const U* upload(const std::vector<U>& v) {
    U* p = alloc<U>(std::max<size_t>(v.size(), 1));
    if (!v.empty()) KS_CUDA(cudaMemcpy(p, v.data(), v.size() * sizeof(U), cudaMemcpyHostToDevice));
    return p;
  }

  const HostGeometry& g_;
  DevTables<float> t_;
  int ns_;
  DeviceArena& arena_;
  StageProfiler& prof_;
  int* err_;
  int N_ = 0, ncols_ = 0, nprojtot_ = 0;
  PlaneNL nl_{};
  std::vector<int> h_pt_off_, h_pt_xy_, h_ent_off_, h_ent_proj_;   // host copies of the plane lists
  std::vector<float> h_ent_beta_;
  bool lists_ready_ = false;
  float2* colbuf1_ = nullptr;
  float2* colbuf2_ = nullptr;
  float* vplane_ = nullptr;
  float2* B_ = nullptr;
  void* Bimg_ = nullptr;             // B_ split into bf16 hi/lo operand tiles
  double2* pout_ = nullptr;
  float2* pf_ = nullptr;
  double2* part_ = nullptr;
  size_t part_elems_ = 0;
  int nch_max_ = 1;
  float* dpartial_ = nullptr;
};

}  // namespace

std::unique_ptr<FusedOps> make_fused_ops(const HostGeometry& g, const DevTables<float>& t, int nstates,
                                         DeviceArena& arena, StageProfiler& prof, int* err) {
  if (!FusedImpl::supported(g.N)) return nullptr;
  return std::unique_ptr<FusedOps>(new FusedImpl(g, t, nstates, arena, prof, err));
}

}  // namespace ks
