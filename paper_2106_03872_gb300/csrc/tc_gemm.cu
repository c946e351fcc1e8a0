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
// MMA tiles are 128 x 256 real (M = 128 rows, N = 256 columns), accumulated in TMEM.  Both
// kernels are warp-specialised: sixteen warps load and split operand chunks into a ring of
// shared-memory stages, one warp issues the MMAs, and stages are handed over with mbarriers
// (the splitters arrive on `full`; tcgen05.commit arrives on `empty` once the MMAs that read
// the stage have completed).  The rotation's M images arrive by bulk copy (TMA).
// Operand tiles use the K-major no-swizzle canonical layout (8-row x 16-byte core
// matrices; LBO = distance between core matrices along K, SBO = along rows).
// Every mbarrier wait is bounded; on expiry the kernel records an error code and returns.
#include <cuda.h>   // driver types only: cuTensorMapEncodeTiled is looked up at run time
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>

#include "kernels.h"

namespace ks {

namespace {

constexpr int TC_M = 128;           // MMA rows
constexpr int TC_N = 256;           // MMA columns
constexpr uint32_t TMEM_COLS = 256;
// rotation: 32 real K per stage (16 states), A hi/lo + three B terms, three stages
constexpr int R_KR = 32;
constexpr int R_KC = R_KR / 2;
constexpr int RA_BYTES = TC_M * R_KR * 2;                 // 8 KB
constexpr int RB_BYTES = TC_N * R_KR * 2;                 // 16 KB
// one CTA: two 128-row tiles of grid coefficients (two TMEM accumulators of 256 columns), so
// each chunk of M images serves 256 rows; A (states, hi/lo per tile) in a 2-deep ring, the
// three M images in a 3-deep ring prefetched two chunks ahead
constexpr int R_TILES = 2;
constexpr int R_SPLIT_WARPS = 16;                            // split X into the A stages
constexpr int R_THREADS = 32 * (R_SPLIT_WARPS + 2);          // + MMA warp + image-copy warp
constexpr int R_A_STAGE = R_TILES * 2 * RA_BYTES;           // 32 KB
constexpr int R_B_STAGE = 3 * RB_BYTES;                      // 48 KB
constexpr int R_NA = 2, R_NB = 3;
constexpr int R_RING = R_NA * R_A_STAGE + R_NB * R_B_STAGE;  // 208 KB
constexpr int R_SMEM = R_RING + 1024;
constexpr uint32_t R_TMEM_COLS = 512;
constexpr long long WAIT_CYCLES = 4000000000LL;          // bound of every mbarrier wait (~2 s)

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

// Bounded wait (by elapsed SM clocks, since a failed try_wait may itself suspend the thread
// for a while); false if the limit expired.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > WAIT_CYCLES) return false;
  return true;
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// Bulk (TMA) copy of `bytes` (multiple of 16, both addresses 16-byte aligned) from global to
// this CTA's shared memory; completion is counted on mbarrier `bar` as transaction bytes.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
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

// x = hi + lo + O(2^-17 |x|) with hi = bf16(x), lo = bf16(x - hi) (as floats).
__device__ __forceinline__ void split1(float x, float& hi, float& lo) {
  hi = __bfloat162float(__float2bfloat16_rn(x));
  lo = x - hi;
}

__device__ __forceinline__ void sts32(uint32_t addr, uint32_t v) {
  asm volatile("st.shared.b32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

__device__ __forceinline__ void sts128(uint32_t addr, uint4 v) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
               : "memory");
}


// ------------------------------------------------------------------------------------------------
// Overlap: part[ks][j][i] = sum_{k in chunk ks} conj(A[i][k]) B[j][k] (FP32), tile 128 (i) x 128 (j).
// Warp roles: warps 0-15 load the FP32 rows of a K-chunk of 16 complex into registers (two
// chunks ahead; rows are only 8-byte aligned when the row length is odd), split them into the
// bf16 hi/lo operand stages and arrive on the stage's `full` barrier; warp 16 issues the MMAs
// and releases the stage through tcgen05.commit on its `empty` barrier.
// ------------------------------------------------------------------------------------------------
constexpr int O_KC = 16;
constexpr int O_KR = 2 * O_KC;
constexpr int O_SPLIT_WARPS = 16;
constexpr int O_THREADS = 32 * (O_SPLIT_WARPS + 1);
constexpr int O_A_BYTES = TC_M * O_KR * 2;                   // 8 KB (hi or lo)
constexpr int O_B_BYTES = TC_N * O_KR * 2;                   // 16 KB
constexpr int O_OP_STAGE = 2 * O_A_BYTES + 2 * O_B_BYTES;    // 48 KB
constexpr int O_NOP = 4;
constexpr int O_RING = O_NOP * O_OP_STAGE;                   // 192 KB
constexpr int O_SMEM = O_RING + 1024;


// PREP: A comes as a pre-split image (k_tc_prep_overlap_a: per 128-row tile and global chunk
// of 16 complex, the hi and lo operand tiles as the split warps would write them) and one
// extra warp copies each chunk's 16 KB with a bulk copy; the split warps handle B alone.
constexpr int O_THREADS_PREP = O_THREADS + 32;
// The PREP form needs fewer registers (54 x 576 threads), so two CTAs share an SM, each with a
// ring of two stages (97 KB): twice the loading warps per SM for the same operand bytes.
constexpr int O_NOP_PREP = 2;
constexpr int O_SMEM_PREP = O_NOP_PREP * O_OP_STAGE + 1024;
template <bool SAME, bool PREP = false>
__global__ void __launch_bounds__(PREP ? O_THREADS_PREP : O_THREADS, PREP ? 2 : 1)
    k_tc_overlap(const float2* __restrict__ A, int lda, const float2* __restrict__ B, int ldb, int m, int n, int K,
                 int kchunk, float2* __restrict__ part, int* __restrict__ err, const uint4* __restrict__ Aimg = nullptr,
                 int nchunks = 0) {
  constexpr int NOP = PREP ? O_NOP_PREP : O_NOP, RING = NOP * O_OP_STAGE;
  extern __shared__ __align__(1024) unsigned char tsm[];
  const uint32_t op0 = smem_u32(tsm);
  uint64_t* bars = reinterpret_cast<uint64_t*>(tsm + RING);
  uint32_t* slot = reinterpret_cast<uint32_t*>(tsm + RING + 128);
  const uint32_t full = smem_u32(bars), empty = full + 8 * NOP, done = empty + 8 * NOP;
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  if (t == 0) {
    for (int i = 0; i < NOP; ++i) {
      mbar_init(full + 8 * i, 32 * O_SPLIT_WARPS + (PREP ? 1 : 0));
      mbar_init(empty + 8 * i, 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (w == 0) tmem_alloc(smem_u32(slot), TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;
  const int i0 = blockIdx.y * TC_M, j0 = blockIdx.x * (TC_N / 2);
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(K, kbeg + kchunk);
  const int nk = (kend - kbeg + O_KC - 1) / O_KC;
  bool ok = true;

  if (w < O_SPLIT_WARPS) {
    // thread (row r, lane-in-row l): complex l, l + 4, l + 8, l + 12 of the chunk for row r
    // of A and complex row r of B, so four lanes read 32 contiguous bytes of a row; each
    // complex becomes one 4-byte (re, im) bf16 pair in K-group u of the tile, and a warp's
    // eight rows fill one core matrix per store
    const int r = t >> 2, l = t & 3, sw = (r >> 2) & 1;
    const bool ra = i0 + r < m, rb = j0 + r < n;
    const float2* pa = A + (size_t)(ra ? i0 + r : 0) * lda;
    const float2* pb = B + (size_t)(rb ? j0 + r : 0) * ldb;
    float2 xa[8], xb[8];                     // [0, 4): A, [4, 8): B
    auto load = [&](int c, float2 (&x)[8]) {
      const int k = kbeg + c * O_KC + l;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (!PREP) x[u] = (ra && k + 4 * u < kend) ? pa[k + 4 * u] : make_float2(0.f, 0.f);
        // SAME: one diagonal tile of A^H A, so B's rows are A's and are loaded once
        x[4 + u] = SAME ? x[u] : ((rb && k + 4 * u < kend) ? pb[k + 4 * u] : make_float2(0.f, 0.f));
      }
    };
    auto chunk = [&](int c, float2 (&x)[8]) {
      const int st = c % NOP;
      if (c >= NOP) {
        ok = mbar_wait_bounded(empty + 8 * st, ((c / NOP) - 1) & 1);
        if (!ok) return;
      }
      const uint32_t oa_hi = op0 + st * O_OP_STAGE, oa_lo = oa_hi + O_A_BYTES;
      const uint32_t ob_hi = oa_hi + 2 * O_A_BYTES, ob_lo = ob_hi + O_B_BYTES;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int kr = 8 * u + 2 * l;        // real K index of the pair
        float h0, l0, h1, l1;
        uint32_t o;
        if (!PREP) {
          split1(x[u].x, h0, l0);
          split1(x[u].y, h1, l1);
          o = tile_off(TC_M, r, kr);
          sts32(oa_hi + o, pack_bf16(h0, h1));
          sts32(oa_lo + o, pack_bf16(l0, l1));
        }
        // B real row 2j <- (re, im), row 2j+1 <- (im, -re)
        split1(x[4 + u].x, h0, l0);
        split1(x[4 + u].y, h1, l1);
        // rows r and r + 4 of a warp write B's two rows in opposite order, so that each store of
        // the warp falls into 32 distinct banks
        const uint32_t e_hi = pack_bf16(h0, h1), e_lo = pack_bf16(l0, l1);
        const uint32_t d_hi = pack_bf16(h1, -h0), d_lo = pack_bf16(l1, -l0);
        o = tile_off(TC_N, 2 * r + sw, kr);
        sts32(ob_hi + o, sw ? d_hi : e_hi);
        sts32(ob_lo + o, sw ? d_lo : e_lo);
        o = tile_off(TC_N, 2 * r + 1 - sw, kr);
        sts32(ob_hi + o, sw ? e_hi : d_hi);
        sts32(ob_lo + o, sw ? e_lo : d_lo);
      }
      fence_proxy_async();
      mbar_arrive(full + 8 * st);
      if (c + 2 < nk) load(c + 2, x);
    };
    if (nk > 0) load(0, xa);
    if (nk > 1) load(1, xb);
    for (int c = 0; c < nk && ok; c += 2) {
      chunk(c, xa);
      if (ok && c + 1 < nk) chunk(c + 1, xb);
    }
  } else if (PREP && w == O_SPLIT_WARPS + 1) {
    // A chunks of this CTA's tile: global chunk kbeg / O_KC + c of the image
    if (lane == 0) {
      const uint4* src = Aimg + ((size_t)blockIdx.y * nchunks + kbeg / O_KC) * (2 * O_A_BYTES / 16);
      for (int c = 0; c < nk; ++c) {
        const int st = c % NOP;
        if (c >= NOP) {
          ok = mbar_wait_bounded(empty + 8 * st, ((c / NOP) - 1) & 1);
          if (!ok) break;
        }
        mbar_expect_tx(full + 8 * st, 2 * O_A_BYTES);
        bulk_g2s(op0 + st * O_OP_STAGE, src + (size_t)c * (2 * O_A_BYTES / 16), 2 * O_A_BYTES, full + 8 * st);
      }
    }
  } else if (w == O_SPLIT_WARPS && lane == 0) {
    constexpr uint32_t idesc = idesc_bf16(TC_M, TC_N);
    constexpr uint32_t a_lbo = TC_M * 16, b_lbo = TC_N * 16;
    for (int c = 0; c < nk; ++c) {
      const int st = c % NOP;
      ok = mbar_wait_bounded(full + 8 * st, (c / NOP) & 1);
      if (!ok) break;
      tc_fence_after();
      const uint32_t oa_hi = op0 + st * O_OP_STAGE, oa_lo = oa_hi + O_A_BYTES;
      const uint32_t ob_hi = oa_hi + 2 * O_A_BYTES, ob_lo = ob_hi + O_B_BYTES;
#pragma unroll
      for (int q = 0; q < O_KR / 16; ++q) {
        const uint32_t ao = 2 * q * a_lbo, bo = 2 * q * b_lbo;
        const uint64_t ahi = smem_desc(oa_hi + ao, a_lbo, 128), alo = smem_desc(oa_lo + ao, a_lbo, 128);
        const uint64_t bhi = smem_desc(ob_hi + bo, b_lbo, 128), blo = smem_desc(ob_lo + bo, b_lbo, 128);
        mma_bf16(tmem, ahi, bhi, idesc, (c == 0 && q == 0) ? 0u : 1u);
        mma_bf16(tmem, ahi, blo, idesc, 1u);
        mma_bf16(tmem, alo, bhi, idesc, 1u);
      }
      mma_commit(empty + 8 * st);
    }
    mma_commit(done);                        // also when nothing was issued
  }
  ok = mbar_wait_bounded(done, 0) && ok;
  ok = __syncthreads_and(ok) != 0;
  if (!ok && t == 0) atomicExch(err, 1);
  tc_fence_after();
  // epilogue (split warps): warp w reads TMEM lanes 32 (w % 4).., columns [64 (w / 4), +64)
  if (ok && w < O_SPLIT_WARPS) {
    const int row = 32 * (w & 3) + lane;
    const int i = i0 + row;
    for (int c0 = 64 * (w >> 2); c0 < 64 * (w >> 2) + 64; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(32 * (w & 3)) << 16) + c0, v);
      // partials column-major (part[z][j][i]): a warp's store covers 32 consecutive i
      if (i < m) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int j = j0 + c0 / 2 + q;
          if (j < n)
            part[((size_t)blockIdx.z * n + j) * m + i] =
                nk > 0 ? make_float2(v[2 * q], v[2 * q + 1]) : make_float2(0.f, 0.f);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (w == 0) tmem_dealloc(tmem, TMEM_COLS);
}

// ------------------------------------------------------------------------------------------------
// The same overlap with the state rows fed by TMA.  Rows are only 8-byte aligned when the row
// length is odd, so one tensor map cannot describe them; the even and the odd rows each form a
// matrix whose row stride (two rows) is a multiple of 16 bytes.  When the row length is odd,
// the odd rows' map starts 8 bytes early, so that its element x + 1 is complex x of the row
// (shift 1).  Per chunk of 16 complex one loader thread issues, per operand and row parity, one
// tiled copy of a 64-row x 18-complex box (coordinates: the chunk's first complex, which is even,
// and the tile's first row / 2) into a raw ring; the split warps read each row's 16 complex from
// shared memory (zero past the CTA's K range; the copies zero-fill outside the operand).  Nothing
// of the rows streams through L1 or registers.  Warps 0-15 split, warp 16 issues the MMAs,
// warp 17 loads, and in the PREP form warp 18 copies A's pre-split operand tiles.
// ------------------------------------------------------------------------------------------------
constexpr int OT_BOX_X = 18, OT_BOX_Y = 64;
constexpr int OT_PITCH = OT_BOX_X * 8;                       // 144 bytes per row of a box
constexpr int OT_BOX_BYTES = OT_PITCH * OT_BOX_Y;            // 9 KB
constexpr int OT_RAW_OPER = 2 * OT_BOX_BYTES;                // both parities of 128 rows
constexpr int OT_NOP = 2;                                    // operand stages

template <bool SAME, bool PREP>
struct OTCfg {
  static constexpr int NOPER = (SAME || PREP) ? 1 : 2;       // operands in the raw ring
  static constexpr int RAW_STAGE = NOPER * OT_RAW_OPER;
  static constexpr int NRAW = NOPER == 1 ? 4 : 3;            // raw stages (72 or 108 KB)
  static constexpr int WARPS = O_SPLIT_WARPS + 2 + (PREP ? 1 : 0);
  static constexpr int THREADS = 32 * WARPS;
  static constexpr int OP_RING = OT_NOP * O_OP_STAGE;        // 96 KB
  static constexpr int RING = OP_RING + NRAW * RAW_STAGE;
  static constexpr int SMEM = RING + 1024;                   // + barriers and the TMEM slot
};

// Tensor maps of up to two operands ([operand][row parity]), the odd rows' shift and the rows
// of each parity.
struct OTMaps {
  CUtensorMap map[2][2];
  int shift[2];
  int rows[2][2];
};

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ float2 lds64(uint32_t addr) {
  float2 v;
  asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr) : "memory");
  return v;
}

template <bool SAME, bool PREP = false>
__global__ void __launch_bounds__(OTCfg<SAME, PREP>::THREADS, 1)
    k_tc_overlap_tma(const __grid_constant__ OTMaps maps, int m, int n, int K, int kchunk, float2* __restrict__ part,
                     int* __restrict__ err, const uint4* __restrict__ Aimg, int nchunks) {
  using CF = OTCfg<SAME, PREP>;
  constexpr int NOP = OT_NOP, NRAW = CF::NRAW, NOPER = CF::NOPER;
  extern __shared__ __align__(1024) unsigned char tsm[];
  const uint32_t op0 = smem_u32(tsm), raw0 = op0 + CF::OP_RING;
  uint64_t* bars = reinterpret_cast<uint64_t*>(tsm + CF::RING);
  uint32_t* slot = reinterpret_cast<uint32_t*>(tsm + CF::RING + 256);
  const uint32_t full = smem_u32(bars), empty = full + 8 * NOP, raw_full = empty + 8 * NOP,
                 raw_empty = raw_full + 8 * NRAW, done = raw_empty + 8 * NRAW;
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  if (t == 0) {
    for (int i = 0; i < NOP; ++i) {
      mbar_init(full + 8 * i, 32 * O_SPLIT_WARPS + (PREP ? 1 : 0));
      mbar_init(empty + 8 * i, 1);
    }
    for (int i = 0; i < NRAW; ++i) {
      mbar_init(raw_full + 8 * i, 1);
      mbar_init(raw_empty + 8 * i, 32 * O_SPLIT_WARPS);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (w == 0) tmem_alloc(smem_u32(slot), TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;
  const int i0 = blockIdx.y * TC_M, j0 = blockIdx.x * (TC_N / 2);
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(K, kbeg + kchunk);
  const int nk = (kend - kbeg + O_KC - 1) / O_KC;
  bool ok = true;
  // raw operand o: B in the PREP form, else A (o = 0) and B (o = 1, not SAME)
  auto first_row = [&](int o) { return (PREP || (!SAME && o == 1)) ? j0 : i0; };
  auto nrows = [&](int o) { return (PREP || (!SAME && o == 1)) ? n : m; };

  if (w < O_SPLIT_WARPS) {
    // thread (row r, lane-in-row l): complex l, l + 4, l + 8, l + 12 of the chunk for row r of
    // each operand (raw box of parity r % 2, box row r / 2); each complex becomes one 4-byte
    // (re, im) bf16 pair in K-group u of the tile, and a warp's eight rows fill one core matrix
    // per store
    const int r = t >> 2, l = t & 3, par = r & 1, sw = (r >> 2) & 1;
    bool rv[NOPER];
    uint32_t rowoff[NOPER];
#pragma unroll
    for (int o = 0; o < NOPER; ++o) {
      rv[o] = first_row(o) + r < nrows(o);
      rowoff[o] = o * OT_RAW_OPER + par * OT_BOX_BYTES + (r >> 1) * OT_PITCH + 8 * (par ? maps.shift[o] : 0);
    }
    for (int c = 0; c < nk && ok; ++c) {
      const int rs = c % NRAW, st = c % NOP;
      ok = mbar_wait_bounded(raw_full + 8 * rs, (c / NRAW) & 1);
      if (ok && c >= NOP) ok = mbar_wait_bounded(empty + 8 * st, ((c / NOP) - 1) & 1);
      if (!ok) break;
      const int nc = min(O_KC, kend - (kbeg + c * O_KC));
      float2 x[NOPER][4];
#pragma unroll
      for (int o = 0; o < NOPER; ++o)
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int k = l + 4 * u;
          x[o][u] = (rv[o] && k < nc) ? lds64(raw0 + rs * CF::RAW_STAGE + rowoff[o] + 8 * k) : make_float2(0.f, 0.f);
        }
      const uint32_t oa_hi = op0 + st * O_OP_STAGE, oa_lo = oa_hi + O_A_BYTES;
      const uint32_t ob_hi = oa_hi + 2 * O_A_BYTES, ob_lo = ob_hi + O_B_BYTES;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int kr = 8 * u + 2 * l;        // real K index of the pair
        float h0, l0, h1, l1;
        uint32_t o;
        if (!PREP) {
          split1(x[0][u].x, h0, l0);
          split1(x[0][u].y, h1, l1);
          o = tile_off(TC_M, r, kr);
          sts32(oa_hi + o, pack_bf16(h0, h1));
          sts32(oa_lo + o, pack_bf16(l0, l1));
        }
        // B real row 2j <- (re, im), row 2j+1 <- (im, -re)
        const float2 xb = x[NOPER - 1][u];
        split1(xb.x, h0, l0);
        split1(xb.y, h1, l1);
        // rows r and r + 4 of a warp write B's two rows in opposite order, so that each store of
        // the warp falls into 32 distinct banks
        const uint32_t e_hi = pack_bf16(h0, h1), e_lo = pack_bf16(l0, l1);
        const uint32_t d_hi = pack_bf16(h1, -h0), d_lo = pack_bf16(l1, -l0);
        o = tile_off(TC_N, 2 * r + sw, kr);
        sts32(ob_hi + o, sw ? d_hi : e_hi);
        sts32(ob_lo + o, sw ? d_lo : e_lo);
        o = tile_off(TC_N, 2 * r + 1 - sw, kr);
        sts32(ob_hi + o, sw ? e_hi : d_hi);
        sts32(ob_lo + o, sw ? e_lo : d_lo);
      }
      fence_proxy_async();
      mbar_arrive(full + 8 * st);
      mbar_arrive(raw_empty + 8 * rs);
    }
  } else if (w == O_SPLIT_WARPS + 1) {
    if (lane == 0) {
      // boxes of this CTA's tiles: row parity p of operand o starts at box row first_row(o) / 2;
      // a box wholly past the parity's rows is not copied (its rows are not read)
      bool has[NOPER][2];
      uint32_t bytes = 0;
#pragma unroll
      for (int o = 0; o < NOPER; ++o)
#pragma unroll
        for (int p = 0; p < 2; ++p) {
          has[o][p] = first_row(o) / 2 < maps.rows[o][p];
          if (has[o][p]) bytes += OT_BOX_BYTES;
        }
      int issued = 0;
      for (int c = 0; c < nk; ++c) {
        const int rs = c % NRAW;
        if (c >= NRAW) {
          ok = mbar_wait_bounded(raw_empty + 8 * rs, ((c / NRAW) - 1) & 1);
          if (!ok) break;
        }
        mbar_expect_tx(raw_full + 8 * rs, bytes);
        const int k0 = kbeg + c * O_KC;
#pragma unroll
        for (int o = 0; o < NOPER; ++o)
#pragma unroll
          for (int p = 0; p < 2; ++p)
            if (has[o][p])
              tma_load_2d(raw0 + rs * CF::RAW_STAGE + o * OT_RAW_OPER + p * OT_BOX_BYTES, &maps.map[o][p], k0,
                          first_row(o) / 2, raw_full + 8 * rs);
        issued = c + 1;
      }
      // copies still in flight land before the CTA exits (the normal path has consumed them all)
      for (int c = max(0, issued - NRAW); c < issued; ++c)
        mbar_wait_bounded(raw_full + 8 * (c % NRAW), (c / NRAW) & 1);
    }
  } else if (PREP && w == O_SPLIT_WARPS + 2) {
    // A chunks of this CTA's tile: global chunk kbeg / O_KC + c of the image
    if (lane == 0) {
      int issued = 0;
      const uint4* src = Aimg + ((size_t)blockIdx.y * nchunks + kbeg / O_KC) * (2 * O_A_BYTES / 16);
      for (int c = 0; c < nk; ++c) {
        const int st = c % NOP;
        if (c >= NOP) {
          ok = mbar_wait_bounded(empty + 8 * st, ((c / NOP) - 1) & 1);
          if (!ok) break;
        }
        mbar_expect_tx(full + 8 * st, 2 * O_A_BYTES);
        bulk_g2s(op0 + st * O_OP_STAGE, src + (size_t)c * (2 * O_A_BYTES / 16), 2 * O_A_BYTES, full + 8 * st);
        issued = c + 1;
      }
      for (int c = max(0, issued - NOP); c < issued; ++c) mbar_wait_bounded(full + 8 * (c % NOP), (c / NOP) & 1);
    }
  } else if (w == O_SPLIT_WARPS && lane == 0) {
    constexpr uint32_t idesc = idesc_bf16(TC_M, TC_N);
    constexpr uint32_t a_lbo = TC_M * 16, b_lbo = TC_N * 16;
    for (int c = 0; c < nk; ++c) {
      const int st = c % NOP;
      ok = mbar_wait_bounded(full + 8 * st, (c / NOP) & 1);
      if (!ok) break;
      tc_fence_after();
      const uint32_t oa_hi = op0 + st * O_OP_STAGE, oa_lo = oa_hi + O_A_BYTES;
      const uint32_t ob_hi = oa_hi + 2 * O_A_BYTES, ob_lo = ob_hi + O_B_BYTES;
#pragma unroll
      for (int q = 0; q < O_KR / 16; ++q) {
        const uint32_t ao = 2 * q * a_lbo, bo = 2 * q * b_lbo;
        const uint64_t ahi = smem_desc(oa_hi + ao, a_lbo, 128), alo = smem_desc(oa_lo + ao, a_lbo, 128);
        const uint64_t bhi = smem_desc(ob_hi + bo, b_lbo, 128), blo = smem_desc(ob_lo + bo, b_lbo, 128);
        mma_bf16(tmem, ahi, bhi, idesc, (c == 0 && q == 0) ? 0u : 1u);
        mma_bf16(tmem, ahi, blo, idesc, 1u);
        mma_bf16(tmem, alo, bhi, idesc, 1u);
      }
      mma_commit(empty + 8 * st);
    }
    mma_commit(done);                        // also when nothing was issued
  }
  ok = mbar_wait_bounded(done, 0) && ok;
  ok = __syncthreads_and(ok) != 0;
  if (!ok && t == 0) atomicExch(err, 1);
  tc_fence_after();
  // epilogue (split warps): warp w reads TMEM lanes 32 (w % 4).., columns [64 (w / 4), +64);
  // partials column-major (part[z][j][i]): a warp's store covers 32 consecutive i
  if (ok && w < O_SPLIT_WARPS) {
    const int i = i0 + 32 * (w & 3) + lane;
    for (int c0 = 64 * (w >> 2); c0 < 64 * (w >> 2) + 64; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(32 * (w & 3)) << 16) + c0, v);
      if (i < m) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int j = j0 + c0 / 2 + q;
          if (j < n)
            part[((size_t)blockIdx.z * n + j) * m + i] =
                nk > 0 ? make_float2(v[2 * q], v[2 * q + 1]) : make_float2(0.f, 0.f);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (w == 0) tmem_dealloc(tmem, TMEM_COLS);
}

// ------------------------------------------------------------------------------------------------
// Rotation: Y[i][k] = sum_j M[i][j] X[j][k].  CTA: 256 grid columns k (two MMA tiles of 128)
// x 128 outputs i.  Mb holds M pre-split into the B-tile images, per (i-tile, j-chunk of 16
// states): the three bf16 terms one after the other.  Per chunk and tile (two K16 steps) the
// MMAs are X_hi M_1 + X_hi M_2 + X_lo M_1 + X_hi M_3.
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ void issue_rotation_tile(uint32_t a, uint32_t b, uint32_t tmem_d, bool first) {
  constexpr uint32_t idesc = idesc_bf16(TC_M, TC_N);
  constexpr uint32_t a_lbo = TC_M * 16, b_lbo = TC_N * 16;
  const uint32_t a_hi = a, a_lo = a + RA_BYTES, b1 = b, b2 = b1 + RB_BYTES, b3 = b2 + RB_BYTES;
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

// Warp roles: warps 0-15 split X (one grid row, 8 states each) into the A stages, warp 16
// issues the MMAs, warp 17 copies each chunk's M images with one bulk copy.  Stage hand-offs
// are mbarriers: a_full (512 arrivals), b_full (transaction bytes), and a_empty / b_empty,
// on which tcgen05.commit arrives when the MMAs that read the stage have completed.
__global__ void __launch_bounds__(R_THREADS, 1)
    k_tc_rotate(const uint4* __restrict__ Mb, int njc, const float2* __restrict__ X, const float2* __restrict__ X2,
                int nin1, int ldx, float2* __restrict__ Y, int ldy, int m, int nin, int K, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char tsm[];
  const uint32_t base = smem_u32(tsm);
  const uint32_t abase = base, bbase = base + R_NA * R_A_STAGE;
  uint64_t* bars = reinterpret_cast<uint64_t*>(tsm + R_RING);
  uint32_t* slot = reinterpret_cast<uint32_t*>(tsm + R_RING + 128);
  const uint32_t bar_base = smem_u32(bars);
  const uint32_t a_full = bar_base, a_empty = bar_base + 8 * R_NA, b_full = bar_base + 16 * R_NA,
                 b_empty = b_full + 8 * R_NB, done = b_empty + 8 * R_NB;
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  if (t == 0) {
    for (int i = 0; i < R_NA; ++i) {
      mbar_init(a_full + 8 * i, 32 * R_SPLIT_WARPS);
      mbar_init(a_empty + 8 * i, 1);
    }
    for (int i = 0; i < R_NB; ++i) {
      mbar_init(b_full + 8 * i, 1);
      mbar_init(b_empty + 8 * i, 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (w == 0) tmem_alloc(smem_u32(slot), R_TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;
  const int k0 = blockIdx.x * (R_TILES * TC_M);
  const int it_i = blockIdx.y;
  const int i0 = it_i * (TC_N / 2);
  bool ok = true;

  if (w < R_SPLIT_WARPS) {
    const int r = t & (R_TILES * TC_M - 1);  // grid coefficient row of the CTA block
    const int tile = r >> 7, tr = r & (TC_M - 1);
    const int jb = t >> 8;                   // which 8 of the 16 states of a chunk
    const int kk = k0 + r;
    // X rows are prefetched into registers two chunks ahead (two register sets, alternating)
    float2 xa[8], xb[8];
    auto load_x = [&](int c, float2 (&xr)[8]) {
      const int jc0 = c * R_KC;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int j = jc0 + 8 * jb + q;
        xr[q] = (j < nin && kk < K) ? (j < nin1 ? X[(size_t)j * ldx + kk] : X2[(size_t)(j - nin1) * ldx + kk])
                                    : make_float2(0.f, 0.f);
      }
    };
    auto chunk = [&](int c, float2 (&xr)[8]) {
      const int st = c % R_NA;
      if (c >= R_NA) {
        ok = mbar_wait_bounded(a_empty + 8 * st, ((c / R_NA) - 1) & 1);
        if (!ok) return;
      }
      const uint32_t sa = abase + st * R_A_STAGE + tile * (2 * RA_BYTES);
      float re[8], im[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        re[q] = xr[q].x;
        im[q] = xr[q].y;
      }
      uint4 hi, lo;
      split8(re, hi, lo);
      uint32_t o = tile_off(TC_M, tr, 8 * jb);
      sts128(sa + o, hi);
      sts128(sa + RA_BYTES + o, lo);
      split8(im, hi, lo);
      o = tile_off(TC_M, tr, 16 + 8 * jb);
      sts128(sa + o, hi);
      sts128(sa + RA_BYTES + o, lo);
      fence_proxy_async();
      mbar_arrive(a_full + 8 * st);
      if (c + 2 < njc) load_x(c + 2, xr);
    };
    if (njc > 0) load_x(0, xa);
    if (njc > 1) load_x(1, xb);
    for (int c = 0; c < njc && ok; c += 2) {
      chunk(c, xa);
      if (ok && c + 1 < njc) chunk(c + 1, xb);
    }
  } else if (w == R_SPLIT_WARPS) {
    if (lane == 0) {
      for (int c = 0; c < njc; ++c) {
        ok = mbar_wait_bounded(a_full + 8 * (c % R_NA), (c / R_NA) & 1) &&
             mbar_wait_bounded(b_full + 8 * (c % R_NB), (c / R_NB) & 1);
        if (!ok) break;
        tc_fence_after();
        const uint32_t a = abase + (c % R_NA) * R_A_STAGE, b = bbase + (c % R_NB) * R_B_STAGE;
#pragma unroll
        for (int q = 0; q < R_TILES; ++q) issue_rotation_tile(a + q * (2 * RA_BYTES), b, tmem + 256 * q, c == 0);
        mma_commit(a_empty + 8 * (c % R_NA));
        mma_commit(b_empty + 8 * (c % R_NB));
      }
      mma_commit(done);                      // also when nothing was issued
    }
  } else if (lane == 0) {
    for (int c = 0; c < njc; ++c) {
      const int st = c % R_NB;
      if (c >= R_NB) {
        ok = mbar_wait_bounded(b_empty + 8 * st, ((c / R_NB) - 1) & 1);
        if (!ok) break;
      }
      mbar_expect_tx(b_full + 8 * st, R_B_STAGE);
      bulk_g2s(bbase + st * R_B_STAGE, Mb + ((size_t)it_i * njc + c) * (R_B_STAGE / 16), R_B_STAGE, b_full + 8 * st);
    }
  }
  ok = mbar_wait_bounded(done, 0) && ok;
  ok = __syncthreads_and(ok) != 0;
  if (!ok && t == 0) atomicExch(err, 1);
  tc_fence_after();
  // epilogue (split warps): warp w reads TMEM lanes 32 (w % 4).., columns [128 (w / 4), +128)
  if (ok && w < R_SPLIT_WARPS) {
    const int q4 = w >> 2;                   // 0..3: tile q4 / 2, half q4 % 2
    const int k = k0 + (q4 >> 1) * TC_M + 32 * (w & 3) + lane;
    for (int c0 = 128 * q4; c0 < 128 * q4 + 128; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(32 * (w & 3)) << 16) + c0, v);
      if (k < K) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int i = i0 + (c0 & 255) / 2 + q;
          if (i < m) Y[(size_t)i * ldy + k] = njc > 0 ? make_float2(v[2 * q], v[2 * q + 1]) : make_float2(0.f, 0.f);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (w == 0) tmem_dealloc(tmem, R_TMEM_COLS);
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

// s + x = hi + err exactly (Knuth's TwoSum); the error terms are summed separately.
__device__ __forceinline__ void two_sum_acc(float& s, float& c, float x) {
  const float t = s + x;
  const float bp = t - s;
  c += (s - (t - bp)) + (x - bp);
  s = t;
}

// out[i][j] = sum_k part[k][j][i]: FP32 partials (exact copies of the TMEM accumulators)
// summed with compensated FP32 arithmetic, so the sum carries about twice FP32's precision
// without the FP64 pipe.  A CTA covers 32 elements e = j m + i (consecutive in the partials);
// warp w takes partials w, w + 8, ...; the eight (sum, error) pairs are combined in a fixed
// order, so the result is deterministic.
__global__ void __launch_bounds__(256) k_reduce_parts_tc(const float2* __restrict__ part, int nks, int m, size_t mn,
                                                         int n, double2* __restrict__ out, float2* __restrict__ out32) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const size_t e = (size_t)blockIdx.x * 32 + lane;
  __shared__ float4 red[8][32];
  float sx = 0.f, cx = 0.f, sy = 0.f, cy = 0.f;
  if (e < mn)
    for (int k = w; k < nks; k += 8) {
      const float2 p = part[(size_t)k * mn + e];
      two_sum_acc(sx, cx, p.x);
      two_sum_acc(sy, cy, p.y);
    }
  red[w][lane] = make_float4(sx, cx, sy, cy);
  __syncthreads();
  if (w == 0 && e < mn) {
    float hx = 0.f, lx = 0.f, hy = 0.f, ly = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float4 r = red[q][lane];
      two_sum_acc(hx, lx, r.x);
      lx += r.y;
      two_sum_acc(hy, ly, r.z);
      ly += r.w;
    }
    const double x = (double)hx + (double)lx, y = (double)hy + (double)ly;
    const size_t o = (e % (size_t)m) * n + e / (size_t)m;             // row-major out[i][j]
    out[o] = make_double2(x, y);
    if (out32) out32[o] = make_float2((float)x, (float)y);
  }
}

// cuTensorMapEncodeTiled, looked up once through the runtime (no link against the driver
// library); null when the driver does not offer it.
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
  static const EncodeTiledFn f = [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return (EncodeTiledFn) nullptr;
    }
    return reinterpret_cast<EncodeTiledFn>(fn);
  }();
  return f;
}

// The row-parity maps of one operand (rows x K, leading dimension ld): false when they cannot
// be formed (operand not 16-byte aligned, or the encoder refuses the shape), in which case the
// overlap runs the register-fed kernel.  The last few operands' maps are kept per host thread.
struct ParityMaps {
  const float2* P = nullptr;
  int ld = 0, rows = 0, K = 0;
  bool ok = false;
  CUtensorMap map[2];
  int shift = 0, prow[2] = {0, 0};
};
const ParityMaps& parity_maps(const float2* P, int ld, int rows, int K) {
  thread_local ParityMaps cache[8];
  thread_local int next = 0;
  for (const ParityMaps& c : cache)
    if (c.P == P && c.ld == ld && c.rows == rows && c.K == K) return c;
  ParityMaps& e = cache[next];
  next = (next + 1) % 8;
  e.P = P;
  e.ld = ld;
  e.rows = rows;
  e.K = K;
  e.ok = false;
  const EncodeTiledFn enc = encode_tiled();
  if (!enc || (reinterpret_cast<uintptr_t>(P) & 15) || rows < 1 || K < 1 || ld < K) return e;
  e.shift = ld & 1;
  for (int p = 0; p < 2; ++p) {
    e.prow[p] = p == 0 ? (rows + 1) / 2 : rows / 2;
    if (e.prow[p] == 0) {                    // no odd rows: never copied
      e.map[1] = e.map[0];
      continue;
    }
    char* base = reinterpret_cast<char*>(const_cast<float2*>(P)) + (p ? 8 * ((size_t)ld - e.shift) : 0);
    const cuuint64_t dims[2] = {(cuuint64_t)K + (p ? e.shift : 0), (cuuint64_t)e.prow[p]};
    const cuuint64_t strides[1] = {(cuuint64_t)16 * ld};
    const cuuint32_t box[2] = {OT_BOX_X, OT_BOX_Y}, estr[2] = {1, 1};
    if (enc(&e.map[p], CU_TENSOR_MAP_DATA_TYPE_INT64, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
        CUDA_SUCCESS)
      return e;
  }
  e.ok = true;
  return e;
}
bool fill_maps(OTMaps& mp, int o, const float2* P, int ld, int rows, int K) {
  const ParityMaps& e = parity_maps(P, ld, rows, K);
  if (!e.ok) return false;
  mp.map[o][0] = e.map[0];
  mp.map[o][1] = e.map[1];
  mp.shift[o] = e.shift;
  mp.rows[o][0] = e.prow[0];
  mp.rows[o][1] = e.prow[1];
  return true;
}

bool g_attr_done = false;
void set_attrs() {
  if (g_attr_done) return;
  KS_CUDA(cudaFuncSetAttribute(k_tc_overlap_tma<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               OTCfg<false, false>::SMEM));
  KS_CUDA(cudaFuncSetAttribute(k_tc_overlap_tma<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               OTCfg<true, false>::SMEM));
  KS_CUDA(cudaFuncSetAttribute(k_tc_overlap_tma<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               OTCfg<false, true>::SMEM));
  KS_CUDA(cudaFuncSetAttribute(k_tc_overlap<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, O_SMEM));
  KS_CUDA(cudaFuncSetAttribute(k_tc_overlap<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, O_SMEM));
  KS_CUDA(cudaFuncSetAttribute(k_tc_overlap<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, O_SMEM_PREP));
  KS_CUDA(cudaFuncSetAttribute(k_tc_rotate, cudaFuncAttributeMaxDynamicSharedMemorySize, R_SMEM));
  g_attr_done = true;
}

// The pre-split image of A for the PREP overlap: thread (tile, chunk, row r, lane l) splits
// the complexes l + 4u (u < 4) of the chunk of row r exactly as the split warps do, into the
// hi and lo tiles of image block (tile, chunk); rows >= m and K >= K are zero.
__global__ void k_tc_prep_overlap_a(const float2* __restrict__ A, int lda, int m, int K, int tiles, int nchunks,
                                    uint32_t* __restrict__ img) {
  const size_t total = (size_t)tiles * nchunks * TC_M * 4;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int l = (int)(e & 3), r = (int)((e >> 2) % TC_M);
    const size_t tc = e / (TC_M * 4);                                 // tile * nchunks + chunk
    const int chunk = (int)(tc % nchunks), tile = (int)(tc / nchunks);
    const int row = tile * TC_M + r;
    uint32_t* blk = img + tc * (2 * O_A_BYTES / 4);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int k = chunk * O_KC + l + 4 * u;
      const float2 x = (row < m && k < K) ? A[(size_t)row * lda + k] : make_float2(0.f, 0.f);
      float h0, l0, h1, l1;
      split1(x.x, h0, l0);
      split1(x.y, h1, l1);
      const uint32_t o = tile_off(TC_M, r, 8 * u + 2 * l) / 4;
      blk[o] = pack_bf16(h0, h1);
      blk[O_A_BYTES / 4 + o] = pack_bf16(l0, l1);
    }
  }
}

}  // namespace

size_t tc_overlap_image_bytes(int m, int K) {
  const int tiles = (m + TC_M - 1) / TC_M, nchunks = (K + O_KC - 1) / O_KC;
  return (size_t)tiles * nchunks * 2 * O_A_BYTES;
}

void tc_overlap_prepare_a(const float2* A, int lda, int m, int K, void* img, cudaStream_t s) {
  const int tiles = (m + TC_M - 1) / TC_M, nchunks = (K + O_KC - 1) / O_KC;
  const size_t total = (size_t)tiles * nchunks * TC_M * 4;
  k_tc_prep_overlap_a<<<(unsigned)std::min<size_t>((total + 255) / 256, 8192), 256, 0, s>>>(
      A, lda, m, K, tiles, nchunks, static_cast<uint32_t*>(img));
  KS_CHECK_LAUNCH();
}

// SMs the overlap kernel spreads its K range over: the device's SMs less four, which the
// block iteration's one-CTA side-stream kernels (factor, Rayleigh-Ritz step) hold while the
// overlaps of the main stream run.  A grid of one CTA per SM would then need a second wave
// for its last CTAs (measured: the 256-projector overlap took 0.24 ms instead of 0.15).
static int sm_count() {
  static const int n = [] {
    int dev = 0, v = 0;
    KS_CUDA(cudaGetDevice(&dev));
    KS_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev));
    return std::max(1, v - 4);
  }();
  return n;
}

size_t tc_overlap_part_elems(int m, int n, bool prepared) {
  const int tm = (m + TC_M - 1) / TC_M, tn = (n + TC_N / 2 - 1) / (TC_N / 2);
  return (size_t)m * n * (size_t)std::max(1, (prepared ? 2 : 1) * sm_count() / (tm * tn));
}

size_t tc_rotation_workspace_bytes(int m, int nin) {
  const int nit = (m + TC_N / 2 - 1) / (TC_N / 2), njc = (nin + R_KC - 1) / R_KC;
  return (size_t)nit * njc * 3 * RB_BYTES;
}

void tc_overlap(const float2* A, int lda, const float2* B, int ldb, int m, int n, int K, double2* part,
                size_t part_elems, double2* out, int* err, cudaStream_t s, float2* out32, const void* Aimg) {
  set_attrs();
  const int tm = (m + TC_M - 1) / TC_M, tn = (n + TC_N / 2 - 1) / (TC_N / 2);
  const bool same = A == B && lda == ldb && m == n && tm == 1 && tn == 1;
  // TMA-fed kernel when the operands' tensor maps can be formed (one CTA per SM)
  OTMaps mp;
  std::memset(&mp, 0, sizeof(mp));
  bool tma;
  if (Aimg)
    tma = fill_maps(mp, 0, B, ldb, n, K);
  else if (same)
    tma = fill_maps(mp, 0, A, lda, m, K);
  else
    tma = fill_maps(mp, 0, A, lda, m, K) && fill_maps(mp, 1, B, ldb, n, K);
  // the register-fed prepared form runs two CTAs per SM
  int ks = std::max(1, (Aimg && !tma ? 2 : 1) * sm_count() / (tm * tn));
  ks = std::min(ks, std::max(1, K / (4 * O_KC)));
  ks = (int)std::min<long>(ks, (long)(part_elems / ((size_t)m * n)));
  if (ks < 1) fail(KS_ERR_ARG, "tc_overlap: partial buffer too small");
  int kchunk = (K + ks - 1) / ks;
  kchunk = (kchunk + O_KC - 1) / O_KC * O_KC;
  ks = (K + kchunk - 1) / kchunk;
  dim3 g(tn, tm, ks);
  float2* p32 = reinterpret_cast<float2*>(part);                      // FP32 partials
  // one output tile of A^H A: both operands are the same rows
  if (tma) {
    if (Aimg)
      k_tc_overlap_tma<false, true><<<g, OTCfg<false, true>::THREADS, OTCfg<false, true>::SMEM, s>>>(
          mp, m, n, K, kchunk, p32, err, static_cast<const uint4*>(Aimg), (K + O_KC - 1) / O_KC);
    else if (same)
      k_tc_overlap_tma<true><<<g, OTCfg<true, false>::THREADS, OTCfg<true, false>::SMEM, s>>>(mp, m, n, K, kchunk, p32,
                                                                                           err, nullptr, 0);
    else
      k_tc_overlap_tma<false><<<g, OTCfg<false, false>::THREADS, OTCfg<false, false>::SMEM, s>>>(
          mp, m, n, K, kchunk, p32, err, nullptr, 0);
  } else if (Aimg)
    k_tc_overlap<false, true><<<g, O_THREADS_PREP, O_SMEM_PREP, s>>>(A, lda, B, ldb, m, n, K, kchunk, p32, err,
                                                                static_cast<const uint4*>(Aimg),
                                                                (K + O_KC - 1) / O_KC);
  else if (same)
    k_tc_overlap<true><<<g, O_THREADS, O_SMEM, s>>>(A, lda, B, ldb, m, n, K, kchunk, p32, err);
  else
    k_tc_overlap<false><<<g, O_THREADS, O_SMEM, s>>>(A, lda, B, ldb, m, n, K, kchunk, p32, err);
  KS_CHECK_LAUNCH();
  const size_t mn = (size_t)m * n;
  k_reduce_parts_tc<<<(unsigned)((mn + 31) / 32), 256, 0, s>>>(p32, ks, m, mn, n, out, out32);
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
  dim3 g((K + R_TILES * TC_M - 1) / (R_TILES * TC_M), nit);
  k_tc_rotate<<<g, R_THREADS, R_SMEM, s>>>(static_cast<const uint4*>(work), njc, X, X2, nin1, ldx, Y, ldy, m, nin, K,
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
