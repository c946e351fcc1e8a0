// Tensor-core (tcgen05, sm_103a) complex GEMMs of the mixed path, split-BF16:
// every FP32 operand x is split into hi = bf16(x) and lo = bf16(x - hi), and each real
// product is accumulated as hi*hi + hi*lo + lo*hi in FP32 in tensor memory (TMEM).  The
// rotation matrix of tc_rotate is split into three bf16 terms (24 significant bits) and
// gets a fourth product, so that its rounding does not bias the norms of rotated states.
//
//   tc_overlap:  out[i][j] = sum_k conj(A[i][k]) B[j][k]       (Gram S, H_sub, projections)
//   tc_rotate:   Y[i][k]   = sum_j M[i][j] X[j][k]             (CholQR and Rayleigh-Ritz rotations;
//                X's rows j >= nin1 may come from a second block X2)
//
// Complex arithmetic as real GEMMs.  Overlap: A is read as a real row of interleaved
// (re, im); B contributes two real rows per complex row, (re, im) and (im, -re), so the
// accumulator column 2j holds Re out[i][j] and column 2j+1 holds Im out[i][j].  Rotation:
// the MMA rows are grid coefficients k, the reduction runs over (j, re|im) and B holds the
// four real blocks of M, so column 2i is Re Y[i][k] and 2i+1 is Im Y[i][k].
//
// One CTA computes a 128 x 256 real tile (M = 128 rows, N = 256 columns) with shared-memory
// rings: all 256 threads load and split the next K-chunk while one thread issues the MMAs
// of the current one; tcgen05.commit arrives on a per-stage mbarrier.
// Operand tiles use the K-major no-swizzle canonical layout (8-row x 16-byte core
// matrices; LBO = distance between core matrices along K, SBO = along rows).
// Every mbarrier wait is bounded; on expiry the kernel records an error code and returns.
#include <cuda_bf16.h>

#include <algorithm>

#include "kernels.h"

namespace ks {

namespace {

constexpr int TC_THREADS = 256;
constexpr int TC_M = 128;           // MMA rows
constexpr int TC_N = 256;           // MMA columns
constexpr uint32_t TMEM_COLS = 256;
// rotation: 32 real K per stage (16 states), A hi/lo + three B terms, three stages
constexpr int R_KR = 32;
constexpr int R_KC = R_KR / 2;
constexpr int RA_BYTES = TC_M * R_KR * 2;                 // 8 KB
constexpr int RB_BYTES = TC_N * R_KR * 2;                 // 16 KB
constexpr int R_STAGE_BYTES = 2 * RA_BYTES + 3 * RB_BYTES; // 64 KB
constexpr int R_NSTAGE = 3;
constexpr int R_SMEM = R_NSTAGE * R_STAGE_BYTES + 1024;
constexpr long WAIT_LIMIT = 1L << 28;                    // spin bound of every mbarrier wait

// ---- PTX wrappers -----------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred P1;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n\t"
      "selp.b32 %0, 1, 0, P1;\n\t}\n"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}

// Bounded wait; false if the limit expired.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  for (long it = 0; it < WAIT_LIMIT; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(ncols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// 16 consecutive 32-bit TMEM columns of this thread's lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// ---- descriptors ------------------------------------------------------------------------------
// Shared-memory matrix descriptor: start >> 4 [0,14), LBO >> 4 [16,30), SBO >> 4 [32,46),
// fixed 0b001 at [46,49), base offset 0, relative LBO, no swizzle.
__host__ __device__ constexpr uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor, kind::f16: D = F32 [4,6), A = B = BF16 [7,10) [10,13), both K-major,
// N >> 3 at [17,23), M >> 4 at [24,29).
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Byte offset of element (row, k) in a K-major no-swizzle tile with R rows:
// core matrix (row/8, k/8) at (k/8) * R * 16 + (row/8) * 128; inside it, row%8 * 16 + k%8 * 2.
__host__ __device__ constexpr uint32_t tile_off(int R, int row, int k) {
  return (uint32_t)((k >> 3) * R * 16 + (row >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

// Split 8 floats into hi and lo bf16 rows of 16 bytes each.
__device__ __forceinline__ void split8(const float (&x)[8], uint4& hi, uint4& lo) {
  float h[8], l[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const __nv_bfloat16 b = __float2bfloat16_rn(x[i]);
    h[i] = __bfloat162float(b);
    l[i] = x[i] - h[i];
  }
  hi = make_uint4(pack_bf16(h[0], h[1]), pack_bf16(h[2], h[3]), pack_bf16(h[4], h[5]), pack_bf16(h[6], h[7]));
  lo = make_uint4(pack_bf16(l[0], l[1]), pack_bf16(l[2], l[3]), pack_bf16(l[4], l[5]), pack_bf16(l[6], l[7]));
}

__device__ __forceinline__ void sts128(uint32_t addr, uint4 v) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
               : "memory");
}

// Common prologue: barriers and TMEM.  Returns the TMEM base address.
__device__ __forceinline__ uint32_t tc_setup(unsigned char* smem, uint32_t& bar0, int ring_bytes, int nstage) {
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + ring_bytes);
  uint32_t* slot = reinterpret_cast<uint32_t*>(smem + ring_bytes + 64);
  bar0 = smem_u32(bars);
  if (threadIdx.x == 0) {
    for (int i = 0; i < nstage; ++i) mbar_init(bar0 + 8 * i, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if ((threadIdx.x >> 5) == 0) tmem_alloc(smem_u32(slot), TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  return *slot;
}

// ------------------------------------------------------------------------------------------------
// Overlap: part[ks][i][j] = sum_{k in chunk ks} conj(A[i][k]) B[j][k], tile 128 (i) x 128 (j).
// Pipeline per K-chunk of 16 complex: cp.async copies raw FP32 rows into a 3-deep ring two
// chunks ahead; all threads split the current chunk into the bf16 operand ring (2 deep);
// one thread issues the MMAs.  Raw rows are padded to 18 complex (144 bytes) so that the
// split pass's 16-byte reads from consecutive rows hit distinct bank groups.
// ------------------------------------------------------------------------------------------------
constexpr int O_KC = 16;
constexpr int O_KR = 2 * O_KC;
constexpr int O_PITCH = 18;                                  // complex per raw row (144 B)
constexpr int O_THREADS = 512;
constexpr int O_RAW_A = TC_M * O_PITCH * 8;                  // 20 KB
constexpr int O_RAW_B = (TC_N / 2) * O_PITCH * 8;            // 20 KB
constexpr int O_RAW_STAGE = O_RAW_A + O_RAW_B;
constexpr int O_NRAW = 3;
constexpr int O_A_BYTES = TC_M * O_KR * 2;                   // 8 KB (hi or lo)
constexpr int O_B_BYTES = TC_N * O_KR * 2;                   // 16 KB
constexpr int O_OP_STAGE = 2 * O_A_BYTES + 2 * O_B_BYTES;    // 48 KB
constexpr int O_NOP = 2;
constexpr int O_RING = O_NRAW * O_RAW_STAGE + O_NOP * O_OP_STAGE;
constexpr int O_SMEM = O_RING + 1024;

__device__ __forceinline__ void cp_async8(uint32_t dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int NPEND> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(NPEND) : "memory");
}

__global__ void __launch_bounds__(O_THREADS, 1)
    k_tc_overlap(const float2* __restrict__ A, int lda, const float2* __restrict__ B, int ldb, int m, int n, int K,
                 int kchunk, double2* __restrict__ part, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char tsm[];
  const uint32_t raw0 = smem_u32(tsm);
  const uint32_t op0 = raw0 + O_NRAW * O_RAW_STAGE;
  const float2* rawp = reinterpret_cast<const float2*>(tsm);
  uint32_t bar0;
  const uint32_t tmem = tc_setup(tsm, bar0, O_RING, O_NOP);
  const int i0 = blockIdx.y * TC_M, j0 = blockIdx.x * (TC_N / 2);
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(K, kbeg + kchunk);
  const int nk = (kend - kbeg + O_KC - 1) / O_KC;
  const int t = threadIdx.x;

  // raw copies of chunk c: 128 rows of A and 128 rows of B, 16 complex each (8-byte copies)
  auto issue_raw = [&](int c) {
    const uint32_t rs = raw0 + (c % O_NRAW) * O_RAW_STAGE;
    const int k0 = kbeg + c * O_KC;
#pragma unroll
    for (int p = 0; p < (TC_M * O_KC) / O_THREADS; ++p) {
      const int idx = p * O_THREADS + t;
      const int r = idx / O_KC, kk = idx - r * O_KC;
      const int k = k0 + kk;
      const bool va = (i0 + r < m) && (k < kend);
      cp_async8(rs + (uint32_t)(r * O_PITCH + kk) * 8, va ? (const void*)(A + (size_t)(i0 + r) * lda + k) : (const void*)A,
                va ? 8u : 0u);
      const bool vb = (j0 + r < n) && (k < kend);
      cp_async8(rs + O_RAW_A + (uint32_t)(r * O_PITCH + kk) * 8,
                vb ? (const void*)(B + (size_t)(j0 + r) * ldb + k) : (const void*)B, vb ? 8u : 0u);
    }
  };

  if (nk > 0) issue_raw(0);
  cp_async_commit();
  if (nk > 1) issue_raw(1);
  cp_async_commit();
  bool ok = true;
  for (int it = 0; it < nk; ++it) {
    if (it + 2 < nk) issue_raw(it + 2);
    cp_async_commit();
    cp_async_wait<2>();            // chunk `it` has landed (this thread's copies)
    __syncthreads();               // ... and every thread's
    const int ost = it % O_NOP;
    if (it >= O_NOP) {
      ok = __syncthreads_and(mbar_wait_bounded(bar0 + 8 * ost, ((it - O_NOP) / O_NOP) & 1)) != 0;
      if (!ok) break;
    }
    const float2* ra = rawp + (size_t)(it % O_NRAW) * (O_RAW_STAGE / 8);
    const float2* rb = ra + O_RAW_A / 8;
    const uint32_t oa_hi = op0 + ost * O_OP_STAGE, oa_lo = oa_hi + O_A_BYTES;
    const uint32_t ob_hi = oa_hi + 2 * O_A_BYTES, ob_lo = ob_hi + O_B_BYTES;
    // A: item (kq, r), 4 complex per item
#pragma unroll
    for (int p = 0; p < (TC_M * (O_KC / 4)) / O_THREADS; ++p) {
      const int item = p * O_THREADS + t;
      const int kq = item / TC_M, r = item - kq * TC_M;
      float x[8];
      const float4* src = reinterpret_cast<const float4*>(ra + r * O_PITCH + 4 * kq);
      const float4 v0 = src[0], v1 = src[1];
      x[0] = v0.x; x[1] = v0.y; x[2] = v0.z; x[3] = v0.w;
      x[4] = v1.x; x[5] = v1.y; x[6] = v1.z; x[7] = v1.w;
      uint4 hi, lo;
      split8(x, hi, lo);
      const uint32_t o = tile_off(TC_M, r, 8 * kq);
      sts128(oa_hi + o, hi);
      sts128(oa_lo + o, lo);
    }
    // B: item (kq, real row e); row 2j <- (re, im), row 2j+1 <- (im, -re)
#pragma unroll
    for (int p = 0; p < (TC_N * (O_KC / 4)) / O_THREADS; ++p) {
      const int item = p * O_THREADS + t;
      const int kq = item / TC_N, e = item - kq * TC_N;
      float x[8];
      const float4* src = reinterpret_cast<const float4*>(rb + (e >> 1) * O_PITCH + 4 * kq);
      const float4 v0 = src[0], v1 = src[1];
      const float y[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (e & 1) {
          x[2 * q] = y[2 * q + 1];
          x[2 * q + 1] = -y[2 * q];
        } else {
          x[2 * q] = y[2 * q];
          x[2 * q + 1] = y[2 * q + 1];
        }
      }
      uint4 hi, lo;
      split8(x, hi, lo);
      const uint32_t o = tile_off(TC_N, e, 8 * kq);
      sts128(ob_hi + o, hi);
      sts128(ob_lo + o, lo);
    }
    fence_proxy_async();
    __syncthreads();
    if (t == 0) {
      tc_fence_after();
      constexpr uint32_t idesc = idesc_bf16(TC_M, TC_N);
      constexpr uint32_t a_lbo = TC_M * 16, b_lbo = TC_N * 16;
#pragma unroll
      for (int s = 0; s < O_KR / 16; ++s) {
        const uint32_t ao = 2 * s * a_lbo, bo = 2 * s * b_lbo;
        const uint64_t ahi = smem_desc(oa_hi + ao, a_lbo, 128), alo = smem_desc(oa_lo + ao, a_lbo, 128);
        const uint64_t bhi = smem_desc(ob_hi + bo, b_lbo, 128), blo = smem_desc(ob_lo + bo, b_lbo, 128);
        mma_bf16(tmem, ahi, bhi, idesc, (it == 0 && s == 0) ? 0u : 1u);
        mma_bf16(tmem, ahi, blo, idesc, 1u);
        mma_bf16(tmem, alo, bhi, idesc, 1u);
      }
      mma_commit(bar0 + 8 * ost);
    }
  }
  cp_async_wait<0>();
  __syncthreads();
  if (ok && nk > 0)
    ok = __syncthreads_and(mbar_wait_bounded(bar0 + 8 * ((nk - 1) % O_NOP), ((nk - 1) / O_NOP) & 1)) != 0;
  if (!ok && t == 0) atomicExch(err, 1);
  tc_fence_after();
  // epilogue: warp w reads TMEM lanes 32*(w%4).., columns [128*(w/4), +128)
  const int w = t >> 5, lane = t & 31;
  const int row = 32 * (w & 3) + lane;
  const int i = i0 + row;
  if (ok) {
    for (int c0 = 64 * (w >> 2); c0 < 64 * (w >> 2) + 64; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(32 * (w & 3)) << 16) + c0, v);
      if (i < m) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int j = j0 + c0 / 2 + q;
          if (j < n)
            part[((size_t)blockIdx.z * m + i) * n + j] =
                nk > 0 ? make_double2((double)v[2 * q], (double)v[2 * q + 1]) : make_double2(0.0, 0.0);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (w == 0) tmem_dealloc(tmem, TMEM_COLS);
}

// ------------------------------------------------------------------------------------------------
// Rotation: Y[i][k] = sum_j M[i][j] X[j][k].  CTA tile: 128 grid columns k x 128 outputs i.
// Mb holds M pre-split into the B-tile images, per (i-tile, j-chunk of 16 states): the
// three bf16 terms one after the other.  Per stage (two K16 steps) the MMAs are
// X_hi M_1 + X_hi M_2 + X_lo M_1 + X_hi M_3.
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ void issue_rotation_stage(uint32_t s, uint32_t tmem_d, bool first) {
  constexpr uint32_t idesc = idesc_bf16(TC_M, TC_N);
  constexpr uint32_t a_lbo = TC_M * 16, b_lbo = TC_N * 16;
  const uint32_t a_hi = s, a_lo = s + RA_BYTES, b1 = s + 2 * RA_BYTES, b2 = b1 + RB_BYTES, b3 = b2 + RB_BYTES;
#pragma unroll
  for (int k = 0; k < R_KR / 16; ++k) {
    const uint32_t ao = 2 * k * a_lbo, bo = 2 * k * b_lbo;
    const uint64_t ah = smem_desc(a_hi + ao, a_lbo, 128), al = smem_desc(a_lo + ao, a_lbo, 128);
    mma_bf16(tmem_d, ah, smem_desc(b1 + bo, b_lbo, 128), idesc, (first && k == 0) ? 0u : 1u);
    mma_bf16(tmem_d, ah, smem_desc(b2 + bo, b_lbo, 128), idesc, 1u);
    mma_bf16(tmem_d, al, smem_desc(b1 + bo, b_lbo, 128), idesc, 1u);
    mma_bf16(tmem_d, ah, smem_desc(b3 + bo, b_lbo, 128), idesc, 1u);
  }
}

__global__ void __launch_bounds__(TC_THREADS, 1)
    k_tc_rotate(const uint4* __restrict__ Mb, int njc, const float2* __restrict__ X, const float2* __restrict__ X2,
                int nin1, int ldx, float2* __restrict__ Y, int ldy, int m, int nin, int K, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char tsm[];
  const uint32_t base = smem_u32(tsm);
  uint32_t bar0;
  const uint32_t tmem = tc_setup(tsm, bar0, R_NSTAGE * R_STAGE_BYTES, R_NSTAGE);
  const int k0 = blockIdx.x * TC_M;
  const int it_i = blockIdx.y;
  const int i0 = it_i * (TC_N / 2);
  const int t = threadIdx.x;
  const int r = t & (TC_M - 1);          // grid coefficient row of the A tile
  const int jb = t >> 7;                 // which 8 of the 16 states of a chunk
  const int kk = k0 + r;
  // pipeline: the three M images of chunk c+1 are copied with cp.async into their stage and
  // the X rows of chunk c+1 are loaded into registers while the MMAs of chunk c run
  float2 xr[8];
  auto load_x = [&](int c) {
    const int jc0 = c * R_KC;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int j = jc0 + 8 * jb + q;
      xr[q] = (j < nin && kk < K) ? (j < nin1 ? X[(size_t)j * ldx + kk] : X2[(size_t)(j - nin1) * ldx + kk])
                                  : make_float2(0.f, 0.f);
    }
  };
  auto issue_b = [&](int c) {
    const uint32_t sb = base + (c % R_NSTAGE) * R_STAGE_BYTES + 2 * RA_BYTES;
    const uint4* src = Mb + ((size_t)it_i * njc + c) * (3 * RB_BYTES / 16);
    for (int v = t; v < 3 * RB_BYTES / 16; v += TC_THREADS) cp_async16(sb + 16 * v, src + v);
  };
  if (njc > 0) {
    issue_b(0);
    load_x(0);
  }
  cp_async_commit();
  bool ok = true;
  for (int it = 0; it < njc; ++it) {
    const int st = it % R_NSTAGE;
    // chunk it+1's stage was last read by the MMAs of chunk it-2
    if (it + 1 < njc && it >= 2) {
      ok = __syncthreads_and(mbar_wait_bounded(bar0 + 8 * ((it + 1) % R_NSTAGE), ((it - 2) / R_NSTAGE) & 1)) != 0;
      if (!ok) break;
    }
    if (it + 1 < njc) issue_b(it + 1);
    cp_async_commit();
    const uint32_t sb = base + st * R_STAGE_BYTES;
    // A: row r = grid coefficient kk; real K: [0,16) re of states jc0.., [16,32) im
    {
      float re[8], im[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        re[q] = xr[q].x;
        im[q] = xr[q].y;
      }
      uint4 hi, lo;
      split8(re, hi, lo);
      uint32_t o = tile_off(TC_M, r, 8 * jb);
      sts128(sb + o, hi);
      sts128(sb + RA_BYTES + o, lo);
      split8(im, hi, lo);
      o = tile_off(TC_M, r, 16 + 8 * jb);
      sts128(sb + o, hi);
      sts128(sb + RA_BYTES + o, lo);
    }
    if (it + 1 < njc) load_x(it + 1);
    cp_async_wait<1>();              // chunk it's images have landed (this thread's copies)
    fence_proxy_async();
    __syncthreads();                 // ... and every thread's, with the A tile stored
    if (t == 0) {
      tc_fence_after();
      issue_rotation_stage(sb, tmem, it == 0);
      mma_commit(bar0 + 8 * st);
    }
  }
  cp_async_wait<0>();
  __syncthreads();
  if (ok && njc > 0)
    ok = __syncthreads_and(mbar_wait_bounded(bar0 + 8 * ((njc - 1) % R_NSTAGE), ((njc - 1) / R_NSTAGE) & 1)) != 0;
  if (!ok && t == 0) atomicExch(err, 1);
  tc_fence_after();
  const int w = t >> 5, lane = t & 31;
  const int row = 32 * (w & 3) + lane;
  const int k = k0 + row;
  if (ok) {
    for (int c0 = 128 * (w >> 2); c0 < 128 * (w >> 2) + 128; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(32 * (w & 3)) << 16) + c0, v);
      if (k < K) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int i = i0 + c0 / 2 + q;
          if (i < m) Y[(size_t)i * ldy + k] = make_float2(v[2 * q], v[2 * q + 1]);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (w == 0) tmem_dealloc(tmem, TMEM_COLS);
}

// Mb images: B row 2i (output Re Y_i) = [Re M_ij | -Im M_ij], row 2i+1 (Im Y_i) = [Im M_ij | Re M_ij]
// over the 16 states of chunk jc (K index kk: kk < 16 -> X_re of state jc*16+kk, else X_im);
// value x = t1 + t2 + t3 with t1 = bf16(x), t2 = bf16(x - t1), t3 = bf16(x - t1 - t2).
// One bf16 term of the three-way split: the nearest bf16 of x, and what it leaves.
__device__ __forceinline__ __nv_bfloat16 split_term(double& x) {
  const __nv_bfloat16 b = __double2bfloat16(x);
  x -= (double)__bfloat162float(b);
  return b;
}
__device__ __forceinline__ __nv_bfloat16 split_term(float& x) {
  const __nv_bfloat16 b = __float2bfloat16_rn(x);
  x -= __bfloat162float(b);                                          // exact in FP32
  return b;
}

template <typename CM>
__global__ void k_tc_prep_rotation(const CM* __restrict__ M, int m, int nin, int nit, int njc,
                                   unsigned char* __restrict__ Mb) {
  using R = decltype(M->x);
  const size_t total = (size_t)nit * njc * TC_N * R_KR;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int kk = (int)(e % R_KR);
    const int row = (int)((e / R_KR) % TC_N);
    const size_t tile = e / ((size_t)R_KR * TC_N);
    const int it_i = (int)(tile / njc), jc = (int)(tile % njc);
    const int i = it_i * (TC_N / 2) + row / 2;
    const int j = jc * R_KC + (kk & (R_KC - 1));
    const int part = kk / R_KC;          // 0: multiplies Re X, 1: Im X
    R x = 0;
    if (i < m && j < nin) {
      const CM v = M[(size_t)i * nin + j];
      if ((row & 1) == 0)
        x = (part == 0 ? v.x : -v.y);
      else
        x = (part == 0 ? v.y : v.x);
    }
    const __nv_bfloat16 t1 = split_term(x);
    const __nv_bfloat16 t2 = split_term(x);
    const __nv_bfloat16 t3 = split_term(x);
    unsigned char* img = Mb + tile * (3 * RB_BYTES);
    const uint32_t o = tile_off(TC_N, row, kk);
    *reinterpret_cast<__nv_bfloat16*>(img + o) = t1;
    *reinterpret_cast<__nv_bfloat16*>(img + RB_BYTES + o) = t2;
    *reinterpret_cast<__nv_bfloat16*>(img + 2 * RB_BYTES + o) = t3;
  }
}

__global__ void k_reduce_parts_tc(const double2* __restrict__ part, int nks, size_t mn, double2* __restrict__ out,
                                  float2* __restrict__ out32) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < mn; e += (size_t)gridDim.x * blockDim.x) {
    double2 s = make_double2(0.0, 0.0);
    for (int k = 0; k < nks; ++k) {
      const double2 p = part[(size_t)k * mn + e];
      s.x += p.x;
      s.y += p.y;
    }
    out[e] = s;
    if (out32) out32[e] = make_float2((float)s.x, (float)s.y);
  }
}

bool g_attr_done = false;
void set_attrs() {
  if (g_attr_done) return;
  KS_CUDA(cudaFuncSetAttribute(k_tc_overlap, cudaFuncAttributeMaxDynamicSharedMemorySize, O_SMEM));
  KS_CUDA(cudaFuncSetAttribute(k_tc_rotate, cudaFuncAttributeMaxDynamicSharedMemorySize, R_SMEM));
  g_attr_done = true;
}

}  // namespace

size_t tc_overlap_part_elems(int m, int n) {
  const int tm = (m + TC_M - 1) / TC_M, tn = (n + TC_N / 2 - 1) / (TC_N / 2);
  return (size_t)m * n * (size_t)std::max(1, 148 / (tm * tn));
}

size_t tc_rotation_workspace_bytes(int m, int nin) {
  const int nit = (m + TC_N / 2 - 1) / (TC_N / 2), njc = (nin + R_KC - 1) / R_KC;
  return (size_t)nit * njc * 3 * RB_BYTES;
}

void tc_overlap(const float2* A, int lda, const float2* B, int ldb, int m, int n, int K, double2* part,
                size_t part_elems, double2* out, int* err, cudaStream_t s, float2* out32) {
  set_attrs();
  const int tm = (m + TC_M - 1) / TC_M, tn = (n + TC_N / 2 - 1) / (TC_N / 2);
  int ks = std::max(1, 148 / (tm * tn));
  ks = std::min(ks, std::max(1, K / (4 * O_KC)));
  ks = (int)std::min<long>(ks, (long)(part_elems / ((size_t)m * n)));
  if (ks < 1) fail(KS_ERR_ARG, "tc_overlap: partial buffer too small");
  int kchunk = (K + ks - 1) / ks;
  kchunk = (kchunk + O_KC - 1) / O_KC * O_KC;
  ks = (K + kchunk - 1) / kchunk;
  dim3 g(tn, tm, ks);
  k_tc_overlap<<<g, O_THREADS, O_SMEM, s>>>(A, lda, B, ldb, m, n, K, kchunk, part, err);
  KS_CHECK_LAUNCH();
  const size_t mn = (size_t)m * n;
  k_reduce_parts_tc<<<(unsigned)std::min<size_t>((mn + 255) / 256, 1024), 256, 0, s>>>(part, ks, mn, out, out32);
  KS_CHECK_LAUNCH();
}

namespace {

template <typename CM>
void prepare_rotation(const CM* M, int m, int nin, void* work, size_t work_bytes, cudaStream_t s) {
  const int nit = (m + TC_N / 2 - 1) / (TC_N / 2), njc = (nin + R_KC - 1) / R_KC;
  if (tc_rotation_workspace_bytes(m, nin) > work_bytes) fail(KS_ERR_ARG, "tc_rotate: workspace too small");
  const size_t total = (size_t)nit * njc * TC_N * R_KR;
  k_tc_prep_rotation<CM><<<(unsigned)std::min<size_t>((total + 255) / 256, 4096), 256, 0, s>>>(
      M, m, nin, nit, njc, static_cast<unsigned char*>(work));
  KS_CHECK_LAUNCH();
}

}  // namespace

void tc_rotate_prepared(const void* work, int nin, const float2* X, const float2* X2, int nin1, int ldx, float2* Y,
                        int ldy, int m, int K, int* err, cudaStream_t s) {
  if (!X2) nin1 = nin;
  set_attrs();
  const int nit = (m + TC_N / 2 - 1) / (TC_N / 2), njc = (nin + R_KC - 1) / R_KC;
  dim3 g((K + TC_M - 1) / TC_M, nit);
  k_tc_rotate<<<g, TC_THREADS, R_SMEM, s>>>(static_cast<const uint4*>(work), njc, X, X2, nin1, ldx, Y, ldy, m, nin, K,
                                            err);
  KS_CHECK_LAUNCH();
}

void tc_rotate_prepare(const float2* M, int m, int nin, void* work, size_t work_bytes, cudaStream_t s) {
  prepare_rotation(M, m, nin, work, work_bytes, s);
}

void tc_rotate(const double2* M, int nin, const float2* X, const float2* X2, int nin1, int ldx, float2* Y, int ldy,
               int m, int K, void* work, size_t work_bytes, int* err, cudaStream_t s) {
  prepare_rotation(M, m, nin, work, work_bytes, s);
  tc_rotate_prepared(work, nin, X, X2, nin1, ldx, Y, ldy, m, K, err, s);
}

}  // namespace ks
