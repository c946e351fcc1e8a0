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
#include "tuner.h"

namespace ks {

namespace {


struct PlaneNL {
  const int* pt_off;     // [N+1] covered points of plane z, sorted by (jy, jx) within the plane
  const int* pt_xy;      // jx*N + jy
  const int* ent_off;    // [npts+1]
  const int* ent_proj;   // first projector row (atom * nproj)
  const float* ent_beta; // [nent][nproj]
  const int* line_off;   // [N][N+1]: points of plane z with y < jy start at pt_off[z] + line_off[z][jy]
  int nproj;
  int cap;               // most covered points of any plane
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
// k_zinv takes ZSB consecutive states per CTA for one block of CT columns and keeps ZNB
// column blocks in shared memory: while one state's block is transformed, the next states'
// coefficients arrive by asynchronous copies (software pipelining hides the load latency that
// one block per CTA left exposed).  Dynamic shared memory: twiddles [N], then the ZNB blocks
// [CT][N + 1].
constexpr int ZSB = 4;
constexpr int ZNB = 3;
template <int N> constexpr size_t zsmem() { return (size_t)(N + ZNB * FCfg<N>::CT * (N + 1)) * sizeof(float2); }

template <int N>
__device__ __forceinline__ void zinv_body(const float2* __restrict__ psi, int nG, const int* __restrict__ col_off,
                                          const int* __restrict__ col_half, int ncols, int nstates,
                                          float2* __restrict__ colbuf, const float2* __restrict__ twg, int yblk) {
  constexpr int CT = FCfg<N>::CT, ld = N + 1, ZT = FCfg<N>::ZT;
  extern __shared__ __align__(16) float2 zsm[];
  float2* tw = zsm;
  float2* sb[ZNB];
#pragma unroll
  for (int i = 0; i < ZNB; ++i) sb[i] = zsm + N + i * CT * ld;
  __shared__ int coff[CT], chalf[CT];
  const int b0 = yblk * ZSB;
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
#pragma unroll
        for (int i = 0; i < ZNB; ++i) sb[i][l * ld + z] = make_float2(0.f, 0.f);
      }
    }
  }
  auto issue = [&](int i) {                                          // state b0 + i -> block i % ZNB
    if (l >= nl) return;
    const float2* col = psi + (size_t)(b0 + i) * nG + g0;
    float2* dst = sb[i % ZNB] + l * ld;
#pragma unroll
    for (int q = 0; q < SLOTS; ++q) {
      const int z = sub + q * TPC;
      if (z < N) {
        const int k = z <= h ? z : (z >= N - h ? z - (N - 2 * h - 1) : -1);
        if (k >= 0) cp_async8(dst + z, col + k);
      }
    }
  };
  // ZNB - 1 states in flight ahead of the one transformed; one commit group per state (empty
  // groups past the last state keep the count)
#pragma unroll
  for (int i = 0; i < ZNB - 1; ++i) {
    if (i < nb) issue(i);
    cp_async_commit();
  }
  for (int i = 0; i < nb; ++i) {
    if (i + ZNB - 1 < nb) issue(i + ZNB - 1);
    cp_async_commit();
    asm volatile("cp.async.wait_group %0;\n" ::"n"(ZNB - 1) : "memory");
    __syncthreads();
    float2* s = sb[i % ZNB];
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
    __syncthreads();                                                  // block i % ZNB free for state i + ZNB
  }
}

template <int N>
__global__ void __launch_bounds__(FCfg<N>::ZT, 2) k_zinv(const float2* __restrict__ psi, int nG, const int* __restrict__ col_off,
                                                      const int* __restrict__ col_half, int ncols, int nstates,
                                                      float2* __restrict__ colbuf, const float2* __restrict__ twg) {
  zinv_body<N>(psi, nG, col_off, col_half, ncols, nstates, colbuf, twg, blockIdx.y);
}

// k_zfwd: one state per CTA (blockIdx.y); the column block arrives by asynchronous copies
// while the state's psi and |G|^2/2 load into registers.  (A ZSB-state pipelined form like
// k_zinv's spilled: the next block's copy addresses and the write-back indices stayed live
// across the transform.)
template <int N>
__device__ __forceinline__ void zfwd_body(const float2* __restrict__ colbuf, const float2* __restrict__ psi,
                                          float2* __restrict__ hpsi, int nG, const int* __restrict__ col_off,
                                          const int* __restrict__ col_half, const float* __restrict__ g2half,
                                          int ncols, float scale, const float2* __restrict__ twg, const TaylorEpi& te,
                                          int b) {
  constexpr int CT = FCfg<N>::CT, ld = N + 1, ZT = FCfg<N>::ZT;
  __shared__ float2 tw[N];
  __shared__ float2 s[CT * ld];
  __shared__ int coff[CT], chalf[CT];
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
      const float2 h = make_float2(u.x * scale + kv[q] * pv[q].x, u.y * scale + kv[q] * pv[q].y);
      const size_t i = off + g0 + k;
      if (!te.skip_h) hpsi[i] = h;
      if (te.nsum) {
        // acc <- base + c[0] w1 + c[1] w2 + c[2] psi + c[3] h, term by term
        const float2 b0 = te.base[i], v1 = te.w1[i], v2 = te.w2[i];
        const float2 tv[4] = {v1, v2, pv[q], h};
        float2 b = b0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          b.x += te.c1[k].x * tv[k].x - te.c1[k].y * tv[k].y;
          b.y += te.c1[k].x * tv[k].y + te.c1[k].y * tv[k].x;
        }
        te.acc1[i] = b;
        if (te.acc2) {
          float2 c = b0;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            c.x += te.c2[k].x * tv[k].x - te.c2[k].y * tv[k].y;
            c.y += te.c2[k].x * tv[k].y + te.c2[k].y * tv[k].x;
          }
          te.acc2[i] = c;
        }
      } else if (te.acc1) {
        // the accumulators of the Taylor series (Eq. 8): acc <- base + a h
        float2 b = te.base_is_psi ? pv[q] : (te.base ? te.base[i] : te.acc1[i]);
        b.x += te.a1.x * h.x - te.a1.y * h.y;
        b.y += te.a1.x * h.y + te.a1.y * h.x;
        te.acc1[i] = b;
        if (te.acc2) {
          float2 c = te.base_is_psi ? pv[q] : (te.base ? te.base[i] : te.acc2[i]);
          c.x += te.a2.x * h.x - te.a2.y * h.y;
          c.y += te.a2.x * h.y + te.a2.y * h.x;
          te.acc2[i] = c;
        }
      }
    }
  }
}

template <int N>
__global__ void __launch_bounds__(FCfg<N>::ZT, 2) k_zfwd(const float2* __restrict__ colbuf, const float2* __restrict__ psi,
                                                      float2* __restrict__ hpsi, int nG, const int* __restrict__ col_off,
                                                      const int* __restrict__ col_half, const float* __restrict__ g2half,
                                                      int ncols, float scale, const float2* __restrict__ twg,
                                                      TaylorEpi te) {
  zfwd_body<N>(colbuf, psi, hpsi, nG, col_off, col_half, g2half, ncols, scale, twg, te, blockIdx.y);
}

// The x-lines (all N) and the y-lines of the rows that hold columns (x in [0, xr] and
// [N - xr, N - 1]) of a plane [x][y] with row pitch N + 1, by the CTA-wide stages of cfft_lines
// (consecutive threads on consecutive lines; with the odd row pitch a warp's 8-byte accesses fall
// on distinct bank pairs in either direction).  Both end with a CTA barrier.
template <int N, int SIGN, class Epi = NoEpi>
__device__ __forceinline__ void x_pass(float2* P, const float2* tw, const Epi& epi = Epi()) {
  cfft_lines<N, FCfg<N>::PT, FCfg<N>::LPC, true, SIGN>(P, N, 1, N + 1, tw, epi);
}

template <int N, int SIGN>
__device__ __forceinline__ void y_pass(float2* P, int xr, const float2* tw) {
  constexpr int ld = N + 1;
  cfft_lines<N, FCfg<N>::PT, FCfg<N>::LPC, true, SIGN>(P, xr + 1, ld, 1, tw);
  if (xr > 0) cfft_lines<N, FCfg<N>::PT, FCfg<N>::LPC, true, SIGN>(P + (N - xr) * ld, xr, ld, 1, tw);
}

// Zero the plane, scatter the columns of one (state, z-plane), inverse y transforms of the
// rows that hold columns.  The first column loads are issued before the plane is cleared, so
// their latency overlaps it.
template <int N>
__device__ __forceinline__ void plane_load_y(float2* P, const float2* __restrict__ colrow, int ncols,
                                             const int* __restrict__ col_xy, int xr, const float2* tw) {
  constexpr int ld = N + 1, PT = FCfg<N>::PT, EARLY = 4;
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
  // y-lines of the rows that hold columns: jx in [0, xr] and [N - xr, N - 1].  With the odd row
  // pitch N + 1 a warp's 8-byte accesses along either direction fall on distinct bank pairs.
  y_pass<N, +1>(P, xr, tw);
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
  constexpr int ld = N + 1, PT = FCfg<N>::PT;
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
  x_pass<N, +1>(P, tw, VMul<N>{Vs});
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
  x_pass<N, -1>(P, tw);
  y_pass<N, -1>(P, xr, tw);
  for (int c = threadIdx.x; c < ncols; c += PT) {
    const int xy = col_xy[c];
    const int jx = xy / N, jy = xy - jx * N;
    colbuf2[row + c] = P[jx * ld + jy];
  }
}

// ---------------------------------------------------------------------------------------------
// Team plane kernel (N = 32, 48, 64, 96, 128): the same H application per (state, z-plane) as k_plane,
// with the line transforms owned by teams of W warps.  A team owns 32 lines, one per lane, so
// a warp's 32 lanes always touch 32 consecutive lines at one element: with the odd row pitch
// N + 1 every shared-memory access is free of bank conflicts along x and along y.  A team's
// stages synchronise on a named barrier of its 32 W threads; the CTA barrier is needed only
// where the transposition between the y and x passes crosses teams.
//
// N = R1 R2.  Inverse transforms: stage A radix R1 over stride-R2 elements (no twiddles), stage B
// radix R2 over stride-R1 elements with twiddles w^(j r), natural order out (Stockham).  Forward
// transforms take the mirrored plan: stage A' radix R2 over stride-R1 elements, stage B' radix R1
// with twiddles.  After the inverse x stage B a thread holds, in registers, exactly the elements
// j + r R1 that the forward x stage A' transforms, so u = V psi + V_NL psi (Eq. 9 add) is formed
// in registers between the two and the x transforms make one shared-memory round trip fewer.
// Rows with |m_x| > x_r hold zeros before the inverse x transform (not loaded) and are not
// needed after the forward one (not stored).  The projector add reads the values of the plane's
// covered points from a list sorted by (y, x) through a per-line bitmap.
// ---------------------------------------------------------------------------------------------
template <int N> struct TPlan {
  static constexpr bool ok = false;
};
template <> struct TPlan<32> { static constexpr bool ok = true; static constexpr int R1 = 8, R2 = 4, W = 4; };
template <> struct TPlan<48> { static constexpr bool ok = true; static constexpr int R1 = 4, R2 = 12, W = 4; };
template <> struct TPlan<64> { static constexpr bool ok = true; static constexpr int R1 = 8, R2 = 8, W = 4; };
template <> struct TPlan<96> { static constexpr bool ok = true; static constexpr int R1 = 8, R2 = 12, W = 4; };
template <> struct TPlan<128> { static constexpr bool ok = true; static constexpr int R1 = 8, R2 = 16, W = 8; };

// Which compiled form of the team plane kernel runs where both would do (the two forms are the
// same code, plane_team_body, and give bitwise the same results; their register allocations
// differ at the 80- and 64-register bounds): at N = 96 the single-cell kernel (no spills) runs
// for every member of a packed H application too, the packed kernel spilling 68 bytes and taking
// 0.683 against 0.614 ms per gs96-sized block; at N = 128 the packed kernel (20 bytes of spills)
// runs for single-cell H applications too, the single-cell one spilling 112 bytes and taking
// 6.75 against 6.44 ms per td128 block.
template <int N> struct PlaneForm {
  static constexpr bool single_per_member = N == 96;
  static constexpr bool packed_for_single = N == 128;
};

template <int N> struct TCfg {
  static constexpr int TEAMS = (N + 31) / 32;
  static constexpr int PT = 32 * TPlan<N>::W * TEAMS;
  static constexpr int PMIN = N >= 128 ? 1 : 2;
  static constexpr int NW = (N + 31) / 32;                // bitmap words per line
};

__device__ __forceinline__ void team_bar(int team, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(1 + team), "r"(nthreads) : "memory");
}

template <int SIGN> __device__ __forceinline__ float2 twiddle(const float2* tw, int t) {
  float2 w = tw[t];
  if (SIGN < 0) w.y = -w.y;
  return w;
}

// Band row g of a plane holds the sphere's columns at |m_y| <= ym[g] only (a column (m_x, m_y)
// exists iff m_x^2 + m_y^2 fits the sphere, a contiguous m_y range per row; ym[g] = -1: none);
// the other elements are read as zeros, so the plane needs no clearing before the scatter.
template <int N> struct ColMask {
  const int* ym;
  __device__ __forceinline__ bool operator()(int g, int y) const {
    const int m = ym[g];
    return y <= m || y >= N - m;
  }
};

// A two-stage transform (R1 then R2, the inverse plan; SIGN selects the exponent) of the lines
// of one team.  Line l at P + off(l), element e at e * KS; stage A reads element e only where
// has(l, e), else zero.  Ends without a barrier: stage B writes back only the elements the same
// thread read.
template <int N, int SIGN, int KS, class Off, class Has>
__device__ __forceinline__ void team_lines(float2* P, int nlines, const Off& off, const float2* tw, const Has& has) {
  using TP = TPlan<N>;
  constexpr int R1 = TP::R1, R2 = TP::R2, W = TP::W, QA = R2 / W, QB = R1 / W;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int team = warp / W, wi = warp - team * W;
  if (team * 32 >= nlines) return;                               // whole team idle (uniform)
  const int l = team * 32 + lane;
  const bool act = l < nlines;
  float2* p = P + off(act ? l : 0);
  {
    float2 v[QA][R1];
#pragma unroll
    for (int q = 0; q < QA; ++q) {
      const int j = wi + W * q;
#pragma unroll
      for (int r = 0; r < R1; ++r)
        v[q][r] = (act && has(l, j + r * R2)) ? p[(j + r * R2) * KS] : make_float2(0.f, 0.f);
      SmallDft<R1, float2>::run(v[q], SIGN);
    }
    team_bar(team, 32 * W);
    if (act) {
#pragma unroll
      for (int q = 0; q < QA; ++q) {
        const int j = wi + W * q;
#pragma unroll
        for (int r = 0; r < R1; ++r) p[(j * R1 + r) * KS] = v[q][r];
      }
    }
    team_bar(team, 32 * W);
  }
  if (act) {
#pragma unroll
    for (int q = 0; q < QB; ++q) {
      const int j = wi + W * q;
      float2 v[R2];
#pragma unroll
      for (int r = 0; r < R2; ++r) v[r] = p[(j + r * R1) * KS];
#pragma unroll
      for (int r = 1; r < R2; ++r) v[r] = cmul(v[r], twiddle<SIGN>(tw, j * r));
      SmallDft<R2, float2>::run(v, SIGN);
#pragma unroll
      for (int r = 0; r < R2; ++r) p[(j + r * R1) * KS] = v[r];
    }
  }
}

// Forward y transform (mirrored plan: R2 then R1) of the band rows of a team.
template <int N, class Off>
__device__ __forceinline__ void team_lines_fwd(float2* P, int nlines, const Off& off, const float2* tw) {
  using TP = TPlan<N>;
  constexpr int R1 = TP::R1, R2 = TP::R2, W = TP::W, QA = R1 / W, QB = R2 / W;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int team = warp / W, wi = warp - team * W;
  if (team * 32 >= nlines) return;
  const int l = team * 32 + lane;
  const bool act = l < nlines;
  float2* p = P + off(act ? l : 0);
  {
    float2 v[QA][R2];
#pragma unroll
    for (int q = 0; q < QA; ++q) {
      const int j = wi + W * q;
#pragma unroll
      for (int r = 0; r < R2; ++r) v[q][r] = act ? p[j + r * R1] : make_float2(0.f, 0.f);
      SmallDft<R2, float2>::run(v[q], -1);
    }
    team_bar(team, 32 * W);
    if (act) {
#pragma unroll
      for (int q = 0; q < QA; ++q) {
        const int j = wi + W * q;
#pragma unroll
        for (int r = 0; r < R2; ++r) p[j * R2 + r] = v[q][r];
      }
    }
    team_bar(team, 32 * W);
  }
  if (act) {
#pragma unroll
    for (int q = 0; q < QB; ++q) {
      const int j = wi + W * q;
      float2 v[R1];
#pragma unroll
      for (int r = 0; r < R1; ++r) v[r] = p[j + r * R2];
#pragma unroll
      for (int r = 1; r < R1; ++r) v[r] = cmul(v[r], twiddle<-1>(tw, j * r));
      SmallDft<R1, float2>::run(v, -1);
#pragma unroll
      for (int r = 0; r < R1; ++r) p[j + r * R2] = v[r];
    }
  }
}

template <int N> struct RowOff {   // band row g -> row x (g <= xr) or g + N - 2 xr - 1, pitch N + 1
  int xr;
  __device__ __forceinline__ int operator()(int g) const { return (g <= xr ? g : g + N - 2 * xr - 1) * (N + 1); }
};
template <int N> struct ColOff {   // x-line = column y of the plane
  __device__ __forceinline__ int operator()(int l) const { return l; }
};

// The x round trip of a team: inverse x transform, u = V psi + the projector add in registers,
// forward x transform.  x-line l (= y) of the plane, element e = x at P[e (N + 1) + l].
template <int N>
__device__ __forceinline__ void team_x_roundtrip(float2* P, int xr, const float* __restrict__ V, const float2* nlv,
                                                 const uint32_t* bits, const int* loff, const float2* tw) {
  using TP = TPlan<N>;
  constexpr int R1 = TP::R1, R2 = TP::R2, W = TP::W, KS = N + 1, NW = TCfg<N>::NW;
  constexpr int QA = R2 / W, QB = R1 / W;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int team = warp / W, wi = warp - team * W;
  const int l = team * 32 + lane;
  const bool act = l < N;
  float2* p = P + (act ? l : 0);
  auto band = [&](int e) { return e <= xr || e >= N - xr; };
  // inverse stage A: radix R1 over e = j + r R2; rows outside the band are zero
  {
    float2 v[QA][R1];
#pragma unroll
    for (int q = 0; q < QA; ++q) {
      const int j = wi + W * q;
#pragma unroll
      for (int r = 0; r < R1; ++r) {
        const int e = j + r * R2;
        v[q][r] = (act && band(e)) ? p[e * KS] : make_float2(0.f, 0.f);
      }
      SmallDft<R1, float2>::run(v[q], +1);
    }
    team_bar(team, 32 * W);
    if (act) {
#pragma unroll
      for (int q = 0; q < QA; ++q) {
        const int j = wi + W * q;
#pragma unroll
        for (int r = 0; r < R1; ++r) p[(j * R1 + r) * KS] = v[q][r];
      }
    }
    team_bar(team, 32 * W);
  }
  // inverse stage B (radix R2, natural order out), pointwise u, forward stage A' (radix R2 on the
  // same elements e = j + r R1)
  {
    // element e = j + R1 r (j < R1, R1 dividing 32) lies in bitmap word (R1 r) / 32 at bit
    // (R1 r mod 32) + j: the word index is a compile-time constant; pre[k] counts the line's points
    // in words < k
    static_assert(32 % R1 == 0, "bitmap word of e = j + R1 r");
    uint32_t wbits[NW];
    int lo = 0;
    if (act) {
      lo = loff[l];
#pragma unroll
      for (int k = 0; k < NW; ++k) wbits[k] = bits[l * NW + k];
    }
    float2 v[QB][R2];
#pragma unroll
    for (int q = 0; q < QB; ++q) {
      const int j = wi + W * q;
      // the potential at this job's elements, requested before the transform so that its L2
      // latency overlaps the arithmetic (all states of a plane read the same V plane)
      float vv[R2];
#pragma unroll
      for (int r = 0; r < R2; ++r) vv[r] = act ? __ldg(V + (j + r * R1) * N + l) : 0.f;
      if (act) {
#pragma unroll
        for (int r = 0; r < R2; ++r) v[q][r] = p[(j + r * R1) * KS];
      } else {
#pragma unroll
        for (int r = 0; r < R2; ++r) v[q][r] = make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int r = 1; r < R2; ++r) v[q][r] = cmul(v[q][r], twiddle<+1>(tw, j * r));
      SmallDft<R2, float2>::run(v[q], +1);
      if (act) {
#pragma unroll
        for (int r = 0; r < R2; ++r) {
          float2 u = make_float2(v[q][r].x * vv[r], v[q][r].y * vv[r]);
          const uint32_t word = wbits[(R1 * r) >> 5];
          const int bit = ((R1 * r) & 31) + j;
          if ((word >> bit) & 1u) {
            int before = lo;                                  // points of this line in earlier words
#pragma unroll
            for (int k = 0; k < (R1 * r) >> 5; ++k) before += __popc(wbits[k]);
            const float2 a = nlv[before + __popc(word & ((1u << bit) - 1u))];
            u.x += a.x;
            u.y += a.y;
          }
          v[q][r] = u;
        }
      }
      SmallDft<R2, float2>::run(v[q], -1);
    }
    team_bar(team, 32 * W);
    if (act) {
#pragma unroll
      for (int q = 0; q < QB; ++q) {
        const int j = wi + W * q;
#pragma unroll
        for (int r = 0; r < R2; ++r) p[(j * R2 + r) * KS] = v[q][r];
      }
    }
    team_bar(team, 32 * W);
  }
  // forward stage B' (radix R1 with twiddles), in place; only the band rows are stored
  if (act) {
#pragma unroll
    for (int q = 0; q < QA; ++q) {
      const int j = wi + W * q;
      float2 v[R1];
#pragma unroll
      for (int r = 0; r < R1; ++r) v[r] = p[(j + r * R2) * KS];
#pragma unroll
      for (int r = 1; r < R1; ++r) v[r] = cmul(v[r], twiddle<-1>(tw, j * r));
      SmallDft<R1, float2>::run(v, -1);
#pragma unroll
      for (int r = 0; r < R1; ++r) {
        const int e = j + r * R2;
        if (band(e)) p[e * KS] = v[r];
      }
    }
  }
}

// Dynamic shared memory: twiddles [N], plane [N][N+1], covered-point values [cap] (rounded up to
// an even count, so that the bitmap is 16-byte aligned), bitmap [N][NW], line offsets [N], row
// column ranges [N].
template <int N> size_t team_smem(int cap) {
  return (size_t)(N + N * (N + 1) + ((cap + 1) & ~1)) * sizeof(float2) +
         (size_t)N * TCfg<N>::NW * sizeof(uint32_t) + 2 * (size_t)N * sizeof(int);
}

// Inputs of the projector add for the team plane kernel: the values sum_{I,l} D Omega^{1/2}
// beta_Il(r) p_Il at the covered points r of every plane, per state (k_nl_values, [state][point],
// points in plane order), the per-plane bitmap of covered points [z][jy][NW] and the per-plane
// y-line offsets of the point list.
struct TeamNL {
  const float2* val;
  const uint32_t* bits;
  const int* pt_off;
  const int* line_off;
  int npts;
};

template <int N>
__device__ __forceinline__ void plane_team_body(const float2* __restrict__ colbuf1, float2* __restrict__ colbuf2,
                                                int ncols, const int* __restrict__ col_xy, int xr,
                                                const int* __restrict__ rowym, const float* __restrict__ vplane,
                                                const TeamNL& nl, int cap_layout, const float2* __restrict__ twg,
                                                int z, int b) {
  constexpr int ld = N + 1, PT = TCfg<N>::PT, NW = TCfg<N>::NW;
  extern __shared__ __align__(16) float2 psm[];
  float2* tw = psm;
  float2* P = tw + N;
  float2* nlv = P + N * ld;
  uint32_t* bits = reinterpret_cast<uint32_t*>(nlv + ((cap_layout + 1) & ~1));
  int* loff = reinterpret_cast<int*>(bits + N * NW);
  int* yms = loff + N;
  // everything the transforms need arrives by asynchronous copies: the columns of this (state,
  // z-plane) into the band rows (no clearing: the inverse y transform reads a row's column range
  // only), the plane's projector values and its bitmap of covered points
  const size_t row = ((size_t)b * N + z) * ncols;
  for (int c = threadIdx.x; c < ncols; c += PT) {
    const int xy = col_xy[c];
    const int jx = xy / N, jy = xy - jx * N;
    cp_async8(P + jx * ld + jy, colbuf1 + row + c);
  }
  if (cap_layout > 0) {
    const int pt0 = nl.pt_off[z], pt1 = nl.pt_off[z + 1];
    const float2* src = nl.val + (size_t)b * nl.npts + pt0;
    for (int q = threadIdx.x; q < pt1 - pt0; q += PT) cp_async8(nlv + q, src + q);
    const uint32_t* bsrc = nl.bits + (size_t)z * N * NW;              // N * NW words: a multiple of 4
    for (int q = threadIdx.x; q < N * NW / 4; q += PT) cp_async16(bits + 4 * q, bsrc + 4 * q);
    for (int e = threadIdx.x; e < N; e += PT) loff[e] = nl.line_off[(size_t)z * (N + 1) + e];
  } else {
    for (int e = threadIdx.x; e < N * NW; e += PT) bits[e] = 0u;
    for (int e = threadIdx.x; e < N; e += PT) loff[e] = 0;
  }
  cp_async_commit();
  for (int t = threadIdx.x; t < N; t += PT) tw[t] = twg[t];
  const int nband = 2 * xr + 1;
  for (int g = threadIdx.x; g < nband; g += PT) yms[g] = rowym[g];
  cp_async_wait_all();
  __syncthreads();
  // inverse y transforms of the band rows
  team_lines<N, +1, 1>(P, nband, RowOff<N>{xr}, tw, ColMask<N>{yms});
  __syncthreads();
  team_x_roundtrip<N>(P, xr, vplane + (size_t)z * N * N, nlv, bits, loff, tw);
  __syncthreads();
  team_lines_fwd<N>(P, nband, RowOff<N>{xr}, tw);
  __syncthreads();
  for (int c = threadIdx.x; c < ncols; c += PT) {
    const int xy = col_xy[c];
    const int jx = xy / N, jy = xy - jx * N;
    colbuf2[row + c] = P[jx * ld + jy];
  }
}

// nlval[b][pt] = sum over the point's sphere entries e (in list order) and projectors q of
// beta_e[q] pf[b][proj_e + q]: the projector add of Eq. 9 at every covered point, per state
// (pf = D Omega^{1/2} p).  One thread per point for NLB consecutive states; with four projectors
// per atom an entry's beta and each state's four projections are 16-byte loads (pf rows and the
// projector offsets are multiples of four).
constexpr int NLB = 8;
template <bool P4>
__global__ void __launch_bounds__(256) k_nl_values(const float2* __restrict__ pf, int nprojtot, int n, PlaneNL nl,
                                                   int npts, float2* __restrict__ nlval) {
  const int pt = blockIdx.x * blockDim.x + threadIdx.x;
  if (pt >= npts) return;
  const int b0 = blockIdx.y * NLB, nb = min(NLB, n - b0);
  float ax[NLB], ay[NLB];
#pragma unroll
  for (int k = 0; k < NLB; ++k) ax[k] = ay[k] = 0.f;
  const int e0 = nl.ent_off[pt], e1 = nl.ent_off[pt + 1];
  for (int e = e0; e < e1; ++e) {
    const float2* pp = pf + (size_t)b0 * nprojtot + nl.ent_proj[e];
    if constexpr (P4) {
      const float4 bt = *reinterpret_cast<const float4*>(nl.ent_beta + (size_t)e * 4);
#pragma unroll
      for (int k = 0; k < NLB; ++k) {
        if (k < nb) {
          const float4 v01 = *reinterpret_cast<const float4*>(pp + (size_t)k * nprojtot);
          const float4 v23 = *reinterpret_cast<const float4*>(pp + (size_t)k * nprojtot + 2);
          ax[k] += bt.x * v01.x;
          ay[k] += bt.x * v01.y;
          ax[k] += bt.y * v01.z;
          ay[k] += bt.y * v01.w;
          ax[k] += bt.z * v23.x;
          ay[k] += bt.z * v23.y;
          ax[k] += bt.w * v23.z;
          ay[k] += bt.w * v23.w;
        }
      }
    } else {
      const float* bt = nl.ent_beta + (size_t)e * nl.nproj;
      for (int q = 0; q < nl.nproj; ++q) {
        const float bq = bt[q];
#pragma unroll
        for (int k = 0; k < NLB; ++k) {
          if (k < nb) {
            const float2 v = pp[(size_t)k * nprojtot + q];
            ax[k] += bq * v.x;
            ay[k] += bq * v.y;
          }
        }
      }
    }
  }
#pragma unroll
  for (int k = 0; k < NLB; ++k)
    if (k < nb) nlval[(size_t)(b0 + k) * npts + pt] = make_float2(ax[k], ay[k]);
}

template <int N>
__global__ void __launch_bounds__(TCfg<N>::PT, TCfg<N>::PMIN)
    k_plane_team(const float2* __restrict__ colbuf1, float2* __restrict__ colbuf2, int ncols,
                 const int* __restrict__ col_xy, int xr, const int* __restrict__ rowym,
                 const float* __restrict__ vplane, TeamNL nl, int cap, const float2* __restrict__ twg) {
  plane_team_body<N>(colbuf1, colbuf2, ncols, col_xy, xr, rowym, vplane, nl, cap, twg, blockIdx.x, blockIdx.y);
}

// ---------------------------------------------------------------------------------------------
// Packed H application of several cells with one grid geometry (fused_apply_h_group): the same
// kernel bodies, launched once over all members' states.  Member m's states are packed rows
// [s0, s0 + n) of the plane and zfwd grids and z-blocks [z0, z0 + ceil(n / ZSB)) of the zinv grid;
// each CTA finds its member by a scan of the descriptor (a kernel parameter, at most GMAX members).
// ---------------------------------------------------------------------------------------------
struct GMember {
  const float2* psi;
  float2* hpsi;
  float2* cb1;
  float2* cb2;
  const float* vplane;
  TeamNL nl;
  TaylorEpi te;
  int cap, n, s0, z0;
};
constexpr int GMAX = 8;
struct GDesc {
  int nm;
  GMember m[GMAX];
};

__device__ __forceinline__ int member_by_state(const GDesc& g, int row) {
  int m = 0;
  while (m + 1 < g.nm && row >= g.m[m + 1].s0) ++m;
  return m;
}
__device__ __forceinline__ int member_by_zblock(const GDesc& g, int row) {
  int m = 0;
  while (m + 1 < g.nm && row >= g.m[m + 1].z0) ++m;
  return m;
}

template <int N>
__global__ void __launch_bounds__(FCfg<N>::ZT, 2) k_zinv_group(const __grid_constant__ GDesc gd, int nG,
                                                            const int* __restrict__ col_off,
                                                            const int* __restrict__ col_half, int ncols,
                                                            const float2* __restrict__ twg) {
  const GMember& M = gd.m[member_by_zblock(gd, blockIdx.y)];
  zinv_body<N>(M.psi, nG, col_off, col_half, ncols, M.n, M.cb1, twg, blockIdx.y - M.z0);
}

template <int N>
__global__ void __launch_bounds__(TCfg<N>::PT, TCfg<N>::PMIN)
    k_plane_team_group(const __grid_constant__ GDesc gd, int ncols, const int* __restrict__ col_xy, int xr,
                       const int* __restrict__ rowym, const float2* __restrict__ twg) {
  const GMember& M = gd.m[member_by_state(gd, blockIdx.y)];
  plane_team_body<N>(M.cb1, M.cb2, ncols, col_xy, xr, rowym, M.vplane, M.nl, M.cap, twg, blockIdx.x,
                     blockIdx.y - M.s0);
}

template <int N>
__global__ void __launch_bounds__(FCfg<N>::ZT, 2) k_zfwd_group(const __grid_constant__ GDesc gd, int nG,
                                                            const int* __restrict__ col_off,
                                                            const int* __restrict__ col_half,
                                                            const float* __restrict__ g2half, int ncols, float scale,
                                                            const float2* __restrict__ twg) {
  const GMember& M = gd.m[member_by_state(gd, blockIdx.y)];
  zfwd_body<N>(M.cb2, M.psi, M.hpsi, nG, col_off, col_half, g2half, ncols, scale, twg, M.te, blockIdx.y - M.s0);
}

// Density partial sums with the team transforms (N = 32, 48, 64, 96, 128): one (z-plane, chunk of
// states) per CTA, states in order.  Per state: the band rows are zeroed, the columns scattered,
// the inverse y transform of the band rows, then the inverse x transform whose stage B leaves
// each thread the elements e = j + r R1 of its x-line in registers; f |u|^2 is added to
// per-thread accumulators (every grid point of the plane belongs to one thread, so each point's
// sum runs over the states in order and needs no atomics).
template <int N>
__global__ void __launch_bounds__(TCfg<N>::PT, TCfg<N>::PMIN)
    k_plane_density_team(const float2* __restrict__ colbuf1, int ncols, const int* __restrict__ col_xy, int xr,
                         const int* __restrict__ rowym, int nstates, int chunk, const double* __restrict__ occ,
                         float scale,
                         float* __restrict__ partial, const float2* __restrict__ twg) {
  using TP = TPlan<N>;
  constexpr int R1 = TP::R1, R2 = TP::R2, W = TP::W, QA = R2 / W, QB = R1 / W;
  constexpr int ld = N + 1, KS = N + 1, PT = TCfg<N>::PT;
  // N = 96 keeps the accumulators in shared memory ([x][y], each point owned by one thread): 24
  // more registers per thread would spill at two CTAs per SM
  constexpr bool ACC_SMEM = N == 96;
  extern __shared__ __align__(16) float2 psm[];
  float2* tw = psm;
  float2* P = tw + N;
  float* accs = reinterpret_cast<float*>(P + N * ld);
  int* yms = reinterpret_cast<int*>(accs + (ACC_SMEM ? N * N : 0));
  const int z = blockIdx.x, ch = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int team = warp / W, wi = warp - team * W;
  const int l = team * 32 + lane;
  const bool act = l < N;
  for (int t = threadIdx.x; t < N; t += PT) tw[t] = twg[t];
  const int nband = 2 * xr + 1;
  for (int g = threadIdx.x; g < nband; g += PT) yms[g] = rowym[g];
  auto band = [&](int e) { return e <= xr || e >= N - xr; };
  float acc[ACC_SMEM ? 1 : QB][ACC_SMEM ? 1 : R2];
  if constexpr (ACC_SMEM) {
    for (int e = threadIdx.x; e < N * N; e += PT) accs[e] = 0.f;
  } else {
#pragma unroll
    for (int q = 0; q < QB; ++q)
#pragma unroll
      for (int r = 0; r < R2; ++r) acc[q][r] = 0.f;
  }
  const int b0 = ch * chunk, b1 = min(nstates, b0 + chunk);
#pragma unroll 1
  for (int b = b0; b < b1; ++b) {
    const float2* src = colbuf1 + ((size_t)b * N + z) * ncols;
    for (int c = threadIdx.x; c < ncols; c += PT) {
      const int xy = col_xy[c];
      const int jx = xy / N, jy = xy - jx * N;
      P[jx * ld + jy] = src[c];
    }
    __syncthreads();
    team_lines<N, +1, 1>(P, nband, RowOff<N>{xr}, tw, ColMask<N>{yms});
    __syncthreads();
    float2* p = P + (act ? l : 0);
    {
      float2 v[QA][R1];
#pragma unroll
      for (int q = 0; q < QA; ++q) {
        const int j = wi + W * q;
#pragma unroll
        for (int r = 0; r < R1; ++r) {
          const int e = j + r * R2;
          v[q][r] = (act && band(e)) ? p[e * KS] : make_float2(0.f, 0.f);
        }
        SmallDft<R1, float2>::run(v[q], +1);
      }
      team_bar(team, 32 * W);
      if (act) {
#pragma unroll
        for (int q = 0; q < QA; ++q) {
          const int j = wi + W * q;
#pragma unroll
          for (int r = 0; r < R1; ++r) p[(j * R1 + r) * KS] = v[q][r];
        }
      }
      team_bar(team, 32 * W);
    }
    const float f = (float)occ[b];
    if (act) {
#pragma unroll
      for (int q = 0; q < QB; ++q) {
        const int j = wi + W * q;
        float2 v[R2];
#pragma unroll
        for (int r = 0; r < R2; ++r) v[r] = p[(j + r * R1) * KS];
#pragma unroll
        for (int r = 1; r < R2; ++r) v[r] = cmul(v[r], twiddle<+1>(tw, j * r));
        SmallDft<R2, float2>::run(v, +1);
#pragma unroll
        for (int r = 0; r < R2; ++r) {
          const float d = f * (v[r].x * v[r].x + v[r].y * v[r].y);
          if constexpr (ACC_SMEM)
            accs[(j + r * R1) * N + l] += d;
          else
            acc[q][r] += d;
        }
      }
    }
    __syncthreads();                                                  // the plane is reused
  }
  float* out = partial + ((size_t)ch * N + z) * N * N;
  if constexpr (ACC_SMEM) {
    for (int e = threadIdx.x; e < N * N; e += PT) out[e] = accs[e] * scale;
  } else if (act) {
#pragma unroll
    for (int q = 0; q < QB; ++q) {
      const int j = wi + W * q;
#pragma unroll
      for (int r = 0; r < R2; ++r) out[(j + r * R1) * N + l] = acc[q][r] * scale;
    }
  }
}

// Real-space planes of the states (forces, Eq. 11, need psi and its gradient on the grid):
// one (state, z-plane) per CTA, the inverse y and x passes of k_plane, then the plane is
// stored contiguously at out[b][z] ([x][y], row pitch N).
template <int N>
__global__ void __launch_bounds__(FCfg<N>::PT, FCfg<N>::PMIN)
    k_plane_inverse(const float2* __restrict__ colbuf1, int ncols, const int* __restrict__ col_xy, int xr,
                    const float2* __restrict__ twg, float2* __restrict__ out) {
  constexpr int ld = N + 1, PT = FCfg<N>::PT;
  extern __shared__ __align__(16) float2 psm[];
  float2* tw = psm;
  float2* P = psm + N;
  const int z = blockIdx.x, b = blockIdx.y;
  for (int t = threadIdx.x; t < N; t += PT) tw[t] = twg[t];
  const size_t row = ((size_t)b * N + z) * ncols;
  plane_load_y<N>(P, colbuf1 + row, ncols, col_xy, xr, tw);
  x_pass<N, +1>(P, tw);
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
  constexpr int ld = N + 1, PT = FCfg<N>::PT;
  extern __shared__ __align__(16) float2 psm[];
  float2* tw = psm;
  float2* P = psm + N;
  float* acc = reinterpret_cast<float*>(P + N * ld);
  const int z = blockIdx.x, b = blockIdx.y;
  for (int t = threadIdx.x; t < N; t += PT) tw[t] = twg[t];
  if (b < nstates) {
    // the y transforms (their first barrier also publishes tw), then the x transforms
    plane_load_y<N>(P, colbuf1 + ((size_t)b * N + z) * ncols, ncols, col_xy, xr, tw);
    x_pass<N, +1>(P, tw, DensSet<N>{acc, (float)occ[b]});
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
  constexpr int ld = N + 1, PT = FCfg<N>::PT;
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
    x_pass<N, +1>(P, tw, DensAcc<N>{acc, (float)occ[b]});
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
            int* err, cudaStream_t setup)
      : g_(g), t_(t), ns_(nstates), arena_(arena), prof_(prof), err_(err), setup_(setup) {
    N_ = g.N;
    ncols_ = g.ncols;
    nprojtot_ = g.natoms * g.nproj;
    const size_t N3 = (size_t)N_ * N_ * N_;
    build_row_ranges();
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
    nch_max_ = std::max((ns_ + density_chunk(0) - 1) / density_chunk(0), (ns_ + density_chunk(1) - 1) / density_chunk(1));
    dpartial_ = alloc<float>((size_t)nch_max_ * N3);
    KS_CUDA(cudaStreamSynchronize(setup_));                           // the uploaded tables have landed
  }

  // The per-cell part of an H application: V re-laid per z-plane and the projections
  // p_Il = sum_G conj(b_Il(G)) c_G of the block (tensor cores), scaled for the plane kernel.
  void pre_h(const float2* psi, int n, const float* v, cudaStream_t s) {
    const size_t N3 = (size_t)N_ * N_ * N_;
    k_to_planes<<<nblk(N3, 256), 256, 0, s>>>(v, N_, vplane_);
    KS_CHECK_LAUNCH();
    if (nprojtot_ > 0) {
      {
        ProfScope ps(prof_, "proj_gemm", s);
        tc_overlap(B_, g_.nG, psi, g_.nG, nprojtot_, n, g_.nG, part_, part_elems_, pout_, err_, s, nullptr, Bimg_);
        const float scale = (float)(g_.D * std::sqrt(g_.omega));
        k_proj_to_states<<<nblk((size_t)nprojtot_ * n, 256), 256, 0, s>>>(pout_, nprojtot_, n, scale, pf_);
        KS_CHECK_LAUNCH();
      }
      if (npts_ > 0 && nlval_) {
        ProfScope ps(prof_, "nl_values", s);
        const dim3 grid((npts_ + 255) / 256, (n + NLB - 1) / NLB);
        if (g_.nproj == 4)
          k_nl_values<true><<<grid, 256, 0, s>>>(pf_, nprojtot_, n, nl_, npts_, nlval_);
        else
          k_nl_values<false><<<grid, 256, 0, s>>>(pf_, nprojtot_, n, nl_, npts_, nlval_);
        KS_CHECK_LAUNCH();
      }
    }
  }

  static bool same_geometry(const FusedImpl* a, const FusedImpl* b) {
    return a->N_ == b->N_ && a->g_.nG == b->g_.nG && a->ncols_ == b->ncols_ && a->g_.xr == b->g_.xr &&
           a->g_.L == b->g_.L && a->g_.ecut == b->g_.ecut;
  }

  // fused_apply_h_group: the members' per-cell parts, then one launch of each kernel per chunk of
  // GMAX members (grids without a team plan: each member alone).
  static void group_apply(const std::vector<FusedGroupItem>& items, cudaStream_t s) {
    if (items.empty()) return;
    FusedImpl* f0 = static_cast<FusedImpl*>(items[0].ops);
    for (const auto& it : items) {
      FusedImpl* f = static_cast<FusedImpl*>(it.ops);
      if (!same_geometry(f0, f)) fail(KS_ERR_ARG, "packed H application: the members' grids differ");
      if (it.n < 1 || it.n > f->ns_) fail(KS_ERR_ARG, "packed H application: member with %d states", it.n);
      f->pre_h(it.psi, it.n, it.v, s);
    }
    f0->dispatch([&](auto tag) { group_launch<decltype(tag)::value>(items, s); });
  }

  template <int N> static void group_launch(const std::vector<FusedGroupItem>& items, cudaStream_t s) {
    FusedImpl* f0 = static_cast<FusedImpl*>(items[0].ops);
    if constexpr (!TPlan<N>::ok) {
      for (const auto& it : items) {
        FusedImpl* f = static_cast<FusedImpl*>(it.ops);
        if (!it.cols_ready) f->zinv(it.psi, it.n, s);
        f->template launch_plane<N>(it.n, f->colbuf1_, f->pf_, s);
        f->template launch_zfwd<N>(it.psi, it.hpsi, it.n, it.te, s);
      }
    } else {
      static bool attr = false;
      if (!attr) {
        KS_CUDA(cudaFuncSetAttribute(k_zinv_group<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zsmem<N>()));
        KS_CUDA(cudaFuncSetAttribute(k_plane_team_group<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)SMEM_MAX));
        attr = true;
      }
      const int ncb = (f0->ncols_ + FCfg<N>::CT - 1) / FCfg<N>::CT;
      for (size_t a = 0; a < items.size(); a += GMAX) {
        GDesc gd{};
        int s0 = 0, z0 = 0;
        size_t smem = 0;
        for (size_t k = a; k < std::min(items.size(), a + GMAX); ++k) {
          const FusedGroupItem& it = items[k];
          FusedImpl* f = static_cast<FusedImpl*>(it.ops);
          GMember& m = gd.m[gd.nm++];
          m.psi = it.psi;
          m.hpsi = it.hpsi;
          m.cb1 = f->colbuf1_;
          m.cb2 = f->colbuf2_;
          m.vplane = f->vplane_;
          m.nl = f->team_nl();
          m.cap = f->team_cap();
          m.te = it.te;
          m.n = it.n;
          m.s0 = s0;
          m.z0 = z0;
          s0 += it.n;
          z0 += (it.n + ZSB - 1) / ZSB;
          smem = std::max(smem, team_smem<N>(m.cap));
        }
        if (smem > SMEM_MAX) fail(KS_ERR_ARG, "packed H application: %zu bytes of shared memory", smem);
        bool cols_ready = true;
        for (size_t k = a; k < std::min(items.size(), a + GMAX); ++k) cols_ready = cols_ready && items[k].cols_ready;
        if (!cols_ready) {
          ProfScope ps(f0->prof_, "zinv", s);
          k_zinv_group<N><<<dim3(ncb, z0), FCfg<N>::ZT, zsmem<N>(), s>>>(gd, f0->g_.nG, f0->t_.col_off,
                                                                         f0->t_.col_half, f0->ncols_, f0->t_.tw);
          KS_CHECK_LAUNCH();
        }
        {
          ProfScope ps(f0->prof_, "plane", s);
          if constexpr (PlaneForm<N>::single_per_member) {
            for (size_t k = a; k < std::min(items.size(), a + GMAX); ++k) {
              FusedImpl* f = static_cast<FusedImpl*>(items[k].ops);
              f->template launch_plane_team_single<N>(items[k].n, s);
            }
          } else {
            k_plane_team_group<N><<<dim3(N, s0), TCfg<N>::PT, smem, s>>>(gd, f0->ncols_, f0->t_.col_xy, f0->g_.xr,
                                                                         f0->rowym_, f0->t_.tw);
            KS_CHECK_LAUNCH();
          }
        }
        {
          ProfScope ps(f0->prof_, "zfwd", s);
          k_zfwd_group<N><<<dim3(ncb, s0), FCfg<N>::ZT, 0, s>>>(gd, f0->g_.nG, f0->t_.col_off, f0->t_.col_half,
                                                                f0->t_.g2half, f0->ncols_,
                                                                (float)(1.0 / ((double)N * N * N)), f0->t_.tw);
          KS_CHECK_LAUNCH();
        }
      }
    }
  }

  void apply_h(const float2* psi, float2* hpsi, int n, const float* v, cudaStream_t s,
               const TaylorEpi* te) override {
    pre_h(psi, n, v, s);
    zinv(psi, n, s);
    {
      ProfScope ps(prof_, "plane", s);
      dispatch([&](auto tag) {
        constexpr int N = decltype(tag)::value;
        launch_plane<N>(n, colbuf1_, pf_, s, plane_variant<N>(n, s));
      });
    }
    {
      ProfScope ps(prof_, "zfwd", s);
      const TaylorEpi none{};
      dispatch([&](auto tag) { launch_zfwd<decltype(tag)::value>(psi, hpsi, n, te ? *te : none, s); });
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
    t_ = t;                                 // the caller has synchronised the engine's streams
    arena_.release(nl_.pt_off);
    arena_.release(nl_.pt_xy);
    arena_.release(nl_.ent_off);
    arena_.release(nl_.ent_proj);
    arena_.release(nl_.ent_beta);
    arena_.release(nl_.line_off);
    arena_.release(nlbits_);
    upload_plane_lists();
    if (nprojtot_ > 0) build_projector_block();
    KS_CUDA(cudaStreamSynchronize(setup_));                           // the new lists have landed
  }

  void density(const float2* psi, int n, const double* occ, float* nout, cudaStream_t s) override {
    zinv(psi, n, s);
    ProfScope ps(prof_, "plane_density", s);
    int variant = 1;
    if (team_density()) {
      static const char* names[2] = {"team", "cta"};
      variant = tune_choice(tune_key("density", n), 2, [&](int c) {
        dispatch([&](auto tag) { launch_density<decltype(tag)::value>(n, occ, s, c); });
      }, s, names);
    }
    dispatch([&](auto tag) { launch_density<decltype(tag)::value>(n, occ, s, variant); });
    const int nch = (n + density_chunk(variant) - 1) / density_chunk(variant);
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
  template <int N> void launch_zfwd(const float2* psi, float2* hpsi, int n, const TaylorEpi& te, cudaStream_t s) {
    dim3 grid((ncols_ + FCfg<N>::CT - 1) / FCfg<N>::CT, n);
    k_zfwd<N><<<grid, FCfg<N>::ZT, 0, s>>>(colbuf2_, psi, hpsi, g_.nG, t_.col_off, t_.col_half, t_.g2half, ncols_,
                                           (float)(1.0 / ((double)N * N * N)), t_.tw, te);
    KS_CHECK_LAUNCH();
  }
  template <int N> static size_t plane_smem() { return (size_t)(N + N * (N + 1)) * sizeof(float2); }
  static constexpr size_t SMEM_MAX = 227 * 1024;
  // Tuned choice of the plane kernel for n states (0: team transforms, 1: CTA-wide stages),
  // where both exist.
  template <int N> int plane_variant(int n, cudaStream_t s) {
    if constexpr (TPlan<N>::ok) {
      if (team_smem<N>(team_cap()) > SMEM_MAX) return 1;
      static const char* names[2] = {"team", "cta"};
      return tune_choice(tune_key("plane", n), 2, [&](int c) { launch_plane<N>(n, colbuf1_, pf_, s, c); }, s,
                         names);
    }
    return 1;
  }
  std::string tune_key(const char* what, int n) const {
    int b = 1;
    while (b < n) b *= 2;
    char buf[96];
    std::snprintf(buf, sizeof(buf), "%s N=%d states<=%d", what, N_, b);
    return buf;
  }

  template <int N> void launch_plane(int n, const float2* cb1, const float2* pf, cudaStream_t s, int variant = 0) {
    if constexpr (TPlan<N>::ok) {
      const size_t smem = team_smem<N>(team_cap());
      if (smem <= SMEM_MAX && variant == 0) {
        if constexpr (PlaneForm<N>::packed_for_single) {
          static bool gattr = false;
          if (!gattr) {
            KS_CUDA(cudaFuncSetAttribute(k_plane_team_group<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)SMEM_MAX));
            gattr = true;
          }
          GDesc gd{};
          gd.nm = 1;
          GMember& m = gd.m[0];
          m.cb1 = const_cast<float2*>(cb1);
          m.cb2 = colbuf2_;
          m.vplane = vplane_;
          m.nl = team_nl();
          m.cap = team_cap();
          m.n = n;
          k_plane_team_group<N><<<dim3(N, n), TCfg<N>::PT, smem, s>>>(gd, ncols_, t_.col_xy, g_.xr, rowym_, t_.tw);
          KS_CHECK_LAUNCH();
          return;
        }
        if (cb1 != colbuf1_) fail(KS_ERR_ARG, "plane kernel: column buffer");
        launch_plane_team_single<N>(n, s);
        return;
      }
    }
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
    k_plane<N><<<grid, FCfg<N>::PT, pf_smem ? with_pf : base, s>>>(cb1, colbuf2_, ncols_, t_.col_xy, g_.xr,
                                                                   vplane_, nl_, pf, nprojtot_, pf_smem, t_.tw);
    KS_CHECK_LAUNCH();
  }
  // The single-cell team plane kernel over n states of this cell's column buffers.
  template <int N> void launch_plane_team_single(int n, cudaStream_t s) {
    if constexpr (TPlan<N>::ok) {
      static bool tattr = false;
      if (!tattr) {
        KS_CUDA(cudaFuncSetAttribute(k_plane_team<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_MAX));
        tattr = true;
      }
      const size_t smem = team_smem<N>(team_cap());
      if (smem > SMEM_MAX) fail(KS_ERR_ARG, "plane kernel: %zu bytes of shared memory for N=%d", smem, N);
      k_plane_team<N><<<dim3(N, n), TCfg<N>::PT, smem, s>>>(colbuf1_, colbuf2_, ncols_, t_.col_xy, g_.xr, rowym_,
                                                            vplane_, team_nl(), team_cap(), t_.tw);
      KS_CHECK_LAUNCH();
    }
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
  // states per density partial: a chunk of states per CTA with the team transforms (about 16
  // chunks, each CTA's partial an N^3 / N plane), else a cluster of DCL states, or a chunk per CTA
  // at N = 128
  bool team_density() const {
    switch (N_) {
      case 32: case 48: case 64: case 96: case 128: return true;
      default: return false;
    }
  }
  // variant 0: the team kernel (about 16 chunks); 1: a cluster of DCL states, or a chunk per CTA
  // at N = 128
  int density_chunk(int variant) const {
    if (variant == 0 && team_density()) return std::max(1, (ns_ + 15) / 16);
    return N_ >= 128 ? std::max(1, std::min(32, (ns_ + 7) / 8)) : DCL;
  }

  template <int N> void launch_density(int n, const double* occ, cudaStream_t s, int variant) {
    const size_t smem = plane_smem<N>() + (size_t)N * N * sizeof(float);
    const int nch = (n + density_chunk(variant) - 1) / density_chunk(variant);
    if constexpr (TPlan<N>::ok) {
      if (variant == 0) {
        static bool attr = false;
        if (!attr) {
          KS_CUDA(cudaFuncSetAttribute(k_plane_density_team<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)SMEM_MAX));
          attr = true;
        }
        const size_t tsmem = plane_smem<N>() + (N == 96 ? (size_t)N * N * sizeof(float) : 0) + N * sizeof(int);
        k_plane_density_team<N><<<dim3(N, nch), TCfg<N>::PT, tsmem, s>>>(colbuf1_, ncols_, t_.col_xy, g_.xr, rowym_, n,
                                                                         density_chunk(0), occ,
                                                                         (float)(1.0 / g_.omega), dpartial_, t_.tw);
        KS_CHECK_LAUNCH();
        return;
      }
    }
    if constexpr (N >= 128) {
      static bool attr = false;
      if (!attr) {
        KS_CUDA(cudaFuncSetAttribute(k_plane_density_chunk<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)SMEM_MAX));
        attr = true;
      }
      k_plane_density_chunk<N><<<dim3(N, nch), FCfg<N>::PT, smem, s>>>(
          colbuf1_, ncols_, t_.col_xy, g_.xr, n, density_chunk(1), occ, (float)(1.0 / g_.omega), dpartial_, t_.tw);
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
    // within a plane, points in (y, x) order, with the offset of each y-line (the team plane
    // kernel finds a point's value by its line's offset and a bitmap of x)
    std::vector<int>& line_off = h_line_off_;
    line_off.assign((size_t)N_ * (N_ + 1), 0);
    nl_cap_ = 0;
    for (int z = 0; z < N_; ++z) {
      std::vector<int>& v = byz[z];
      std::stable_sort(v.begin(), v.end(), [&](int a, int b) {
        const int xa = g.cov_idx[a] / N_, xb = g.cov_idx[b] / N_;       // jx*N + jy
        return (xa % N_) != (xb % N_) ? (xa % N_) < (xb % N_) : (xa / N_) < (xb / N_);
      });
      int* lo = line_off.data() + (size_t)z * (N_ + 1);
      for (int c : v) lo[(g.cov_idx[c] / N_) % N_ + 1]++;
      for (int y = 0; y < N_; ++y) lo[y + 1] += lo[y];
      nl_cap_ = std::max(nl_cap_, (int)v.size());
      for (int c : v) {
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
    nl_.line_off = upload(h_line_off_);
    nl_.nproj = g_.nproj;
    nl_.cap = nl_cap_;
    // per-plane bitmap of the covered points ([z][jy][NW], bit jx) for the team plane kernel, and
    // the projector values of every covered point per state (grown when the atoms move)
    const int NW = (N_ + 31) / 32;
    std::vector<uint32_t> bits((size_t)N_ * N_ * NW, 0u);
    for (int z = 0; z < N_; ++z)
      for (int pt = h_pt_off_[z]; pt < h_pt_off_[z + 1]; ++pt) {
        const int jx = h_pt_xy_[pt] / N_, jy = h_pt_xy_[pt] % N_;
        bits[((size_t)z * N_ + jy) * NW + (jx >> 5)] |= 1u << (jx & 31);
      }
    nlbits_ = upload(bits);
    npts_ = h_pt_off_[N_];
    if (nprojtot_ > 0 && (size_t)npts_ > nlval_pts_) {
      if (nlval_) arena_.release(nlval_);
      nlval_pts_ = (size_t)npts_ + npts_ / 8;                      // room for moves that cover more points
      nlval_ = alloc<float2>((size_t)ns_ * nlval_pts_);
    }
  }

  // ym[g] of band row g (m_x = g for g <= xr, else g - 2 xr - 1): the largest |m_y| of the
  // sphere's columns in that row, whose columns are exactly |m_y| <= ym[g]
  void build_row_ranges() {
    const int nband = 2 * g_.xr + 1;
    std::vector<int> ym(nband, -1), cnt(nband, 0);
    for (int xy : g_.col_xy) {
      const int jx = xy / N_, jy = xy % N_;
      const int mx = jx < (N_ + 1) / 2 ? jx : jx - N_, my = jy < (N_ + 1) / 2 ? jy : jy - N_;
      const int gr = mx >= 0 ? mx : mx + nband;
      if (gr < 0 || gr >= nband) fail(KS_ERR_ARG, "plane kernel: column outside the band (m_x = %d)", mx);
      ym[gr] = std::max(ym[gr], std::abs(my));
      cnt[gr]++;
    }
    for (int gr = 0; gr < nband; ++gr)
      if (cnt[gr] != (ym[gr] < 0 ? 0 : 2 * ym[gr] + 1) || 2 * ym[gr] + 1 > N_)
        fail(KS_ERR_ARG, "plane kernel: the columns of band row %d are not one m_y range", gr);
    rowym_ = upload(ym);
  }
  TeamNL team_nl() const { return TeamNL{nlval_, nlbits_, nl_.pt_off, nl_.line_off, npts_}; }
  int team_cap() const { return nprojtot_ > 0 ? nl_cap_ : 0; }

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
    // temporaries from the engine's arena (a server's pool when there is one), returned below
    const float2* tw = t_.tw;                                         // (cos, sin)(2 pi t / N), FP32
    float* dbox = alloc<float>(box.size());
    int* dlo = alloc<int>(std::max<size_t>(1, lo.size()));
    float2* T1 = alloc<float2>((size_t)chunk * B * B * M);
    float2* T2 = alloc<float2>((size_t)chunk * B * M * M);
    KS_CUDA(cudaMemcpyAsync(dbox, box.data(), box.size() * sizeof(float), cudaMemcpyHostToDevice, setup_));
    KS_CUDA(cudaMemcpyAsync(dlo, lo.data(), lo.size() * sizeof(int), cudaMemcpyHostToDevice, setup_));
    const float scale = (float)(std::sqrt(g.omega) / ((double)N * N * N));
    for (int r0 = 0; r0 < nprojtot_; r0 += chunk) {                   // r0: a multiple of np
      const int nr = std::min(chunk, nprojtot_ - r0);
      const int* clo = dlo + 3 * (r0 / np);
      k_box_dft_z<<<nblk((size_t)nr * B * B * M, 256), 256, 0, setup_>>>(dbox + (size_t)r0 * B * B * B, clo, np, nr,
                                                                          B, xr, N, tw, T1);
      KS_CHECK_LAUNCH();
      k_box_dft_y<<<nblk((size_t)nr * B * M * M, 256), 256, 0, setup_>>>(T1, clo, np, nr, B, xr, N, tw, T2);
      KS_CHECK_LAUNCH();
      k_box_dft_x<<<nblk((size_t)nr * g.nG, 256), 256, 0, setup_>>>(T2, clo, t_.gidx, np, nr, B, xr, N, g.nG, scale,
                                                                    tw, B_ + (size_t)r0 * g.nG);
      KS_CHECK_LAUNCH();
    }
    tc_overlap_prepare_a(B_, g.nG, nprojtot_, g.nG, Bimg_, setup_);    // the operand split once
    KS_CUDA(cudaStreamSynchronize(setup_));                            // the temporaries are idle
    arena_.release(dbox);
    arena_.release(dlo);
    arena_.release(T1);
    arena_.release(T2);
  }

  template <typename U> U* alloc(size_t n) { return static_cast<U*>(arena_.alloc(n * sizeof(U))); }
  template <typename U> const U* upload(const std::vector<U>& v) {
    U* p = alloc<U>(std::max<size_t>(v.size(), 1));
    if (!v.empty()) KS_CUDA(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(U), cudaMemcpyHostToDevice, setup_));
    return p;
  }

  const HostGeometry& g_;
  DevTables<float> t_;
  int ns_;
  DeviceArena& arena_;
  StageProfiler& prof_;
  int* err_;
  cudaStream_t setup_;
  int N_ = 0, ncols_ = 0, nprojtot_ = 0;
  PlaneNL nl_{};
  std::vector<int> h_pt_off_, h_pt_xy_, h_ent_off_, h_ent_proj_;   // host copies of the plane lists
  std::vector<float> h_ent_beta_;
  std::vector<int> h_line_off_;       // [N][N+1] per-plane y-line offsets of the covered points
  int nl_cap_ = 0;                    // most covered points of any plane
  bool lists_ready_ = false;
  float2* colbuf1_ = nullptr;
  float2* colbuf2_ = nullptr;
  float* vplane_ = nullptr;
  float2* B_ = nullptr;
  void* Bimg_ = nullptr;             // B_ split into bf16 hi/lo operand tiles
  double2* pout_ = nullptr;
  float2* pf_ = nullptr;
  const int* rowym_ = nullptr;       // [2 xr + 1] column range of each band row
  const uint32_t* nlbits_ = nullptr; // [N][N][NW] covered points of each plane
  float2* nlval_ = nullptr;          // [ns][nlval_pts_] projector values of the covered points
  size_t nlval_pts_ = 0;
  int npts_ = 0;                     // covered points of all planes
  double2* part_ = nullptr;
  size_t part_elems_ = 0;
  int nch_max_ = 1;
  float* dpartial_ = nullptr;
};

}  // namespace

void fused_apply_h_group(const std::vector<FusedGroupItem>& items, cudaStream_t s) {
  FusedImpl::group_apply(items, s);
}

bool fused_same_geometry(const FusedOps* a, const FusedOps* b) {
  return FusedImpl::same_geometry(static_cast<const FusedImpl*>(a), static_cast<const FusedImpl*>(b));
}

std::unique_ptr<FusedOps> make_fused_ops(const HostGeometry& g, const DevTables<float>& t, int nstates,
                                         DeviceArena& arena, StageProfiler& prof, int* err, cudaStream_t setup) {
  if (!FusedImpl::supported(g.N)) return nullptr;
  return std::unique_ptr<FusedOps>(new FusedImpl(g, t, nstates, arena, prof, err, setup));
}

}  // namespace ks
