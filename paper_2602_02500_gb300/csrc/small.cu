// Algorithm 1 (Sec. 2.4) for matrices with h <= 128, one CTA per matrix,
// entirely on chip (sm_103a).
//
// A matrix this small fits one 128 x 128 tensor-core tile, so the tiled
// passes (one launch per pass, every intermediate through HBM, h padded to
// 256) spend their time on launches and padding.  Here one CTA runs the
// whole chain:
//   Gram      T_0 = A A^T on tcgen05 (M = N = 128, K = w streamed by TMA),
//             accumulator in TMEM;
//   scalars   o = ||T_0||_F (or ||A||_F^2), tr T_0, 1/o, 1/sqrt(o), the
//             D-basis identity weight c_0 = 1 + sum_l w_l (FP64);
//   squarings D_1 = T_0 / o, D_{l+1} = 2 D_l - D_l^2 (l = 1..L-1): D_l lives
//             in shared memory as the FP16 operand of the next product (hi,
//             or hi + lo for the leading squarings of the mixed precision,
//             three products hi hi + hi lo + lo hi) and in FP32 in the
//             epilogue warps' registers; P = c_0 I - sum_l w_l D_l in FP32
//             in TMEM (columns 256..383) beside the squarings' two
//             accumulators (columns 0..127 and 128..255, in turn);
//   product   Y = P A / sqrt(o) with P as BF16 hi + lo in shared memory and
//             A streamed again in 256-column tiles, written in M's shape.
// Rows and columns past h are zero (TMA zero fill), so they drop out of
// every product.
//
// Warp roles (320 threads): warp 0 TMA producer, warp 1 TMEM owner and MMA
// issuer, warps 2..9 epilogue (two per TMEM lane quadrant; each thread owns
// one row and 64 columns of the 128 x 128 intermediates, 32 in each K
// block).  Every wait is
// bounded as in the tiled kernels (ptx.cuh): a timeout records
// IFNSO_DEV_TIMEOUT for the matrix, lets issued copies and products land,
// frees TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "common.cuh"
#include "ptx.cuh"

namespace ifnso {
namespace {

constexpr int kThreads = 320;
constexpr uint32_t kOpBuf = 128 * 128 * 2;        // one 128 x 128 16-bit operand: two 64-wide K blocks
constexpr uint32_t kKBlock = 128 * 64 * 2;        // 16 KB: 128 rows x 64 K (128-byte swizzled rows)
constexpr uint32_t kApplyStage = 256 * 64 * 2;    // 32 KB: 256 B-operand rows x 64 K
constexpr uint32_t kRing = 4 * kApplyStage;       // 128 KB, shared by the Gram (8 x 16 KB) and product (4 x 32 KB) rings
constexpr int kGramStages = static_cast<int>(kRing / kKBlock);
constexpr int kApplyStages = static_cast<int>(kRing / kApplyStage);
constexpr uint32_t kTail = 1024;  // barriers, TMEM slot, abort flag, partial sums, coefficients
constexpr uint32_t kStg = 8 * 2048;  // one 32 x 32 BF16 output staging block per epilogue warp
constexpr uint32_t kSmem = 1024 + kRing + 2 * kOpBuf + kTail + kStg;
constexpr int kDevTimeout = 4, kDevZero = 1, kDevNonFinite = 2;

// Barrier slots (8 bytes each) after the buffers.
enum Bar {
  kGFull = 0,
  kGEmpty = kGFull + kGramStages,
  kAFull = kGEmpty + kGramStages,
  kAEmpty = kAFull + kApplyStages,
  kTFull = kAEmpty + kApplyStages,  // Gram / squaring accumulator ready (one phase per product)
  kDReady,                          // K block 0 of D_1 .. D_{L-1} written (8 epilogue warps per phase)
  kDReady1,                         // K block 1 of the same
  kPReady,                          // P written (8 epilogue warps)
  kGDone,                           // the Gram's products have read their ring stages
  kT2Full,                          // product accumulators 0, 1 ready
  kT2Empty = kT2Full + 2,           // product accumulators 0, 1 drained (8 warps each)
  kDrain = kT2Empty + 2,
  kNumBars
};
static_assert(kNumBars * 8 + 8 + 8 * 8 + 32 * 8 + 8 <= kTail,
              "barriers, TMEM slot, abort flag, 8 partial sums, 32 coefficients, 2 scalars");

__device__ __forceinline__ uint32_t sw128_off(int row, int chunk) {
  // byte offset of 16-byte chunk `chunk` (0..7) of row `row` in a 128-byte
  // swizzled K-major block (8-row groups 1024 bytes apart)
  return static_cast<uint32_t>((row >> 3) * 1024 + (row & 7) * 128 + ((chunk ^ (row & 7)) << 4));
}

template <typename T>
__device__ __forceinline__ uint4 pack8(const float* x);
template <>
__device__ __forceinline__ uint4 pack8<__half>(const float* x) {
  uint4 u;
  __half2* h = reinterpret_cast<__half2*>(&u);
#pragma unroll
  for (int t = 0; t < 4; ++t) h[t] = __floats2half2_rn(x[2 * t], x[2 * t + 1]);
  return u;
}
template <>
__device__ __forceinline__ uint4 pack8<__nv_bfloat16>(const float* x) {
  uint4 u;
  __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&u);
#pragma unroll
  for (int t = 0; t < 4; ++t) h[t] = __floats2bfloat162_rn(x[2 * t], x[2 * t + 1]);
  return u;
}

// This warp's 32 x 32 block of Y (lane t: row r0 + t, columns c0 .. c0 + 31
// in y) to out (BF16, leading dimension ld) through the warp's 2 KB staging
// buffer, so that each store instruction writes 64-byte row pieces of 8 rows
// (not 16 bytes in each of 32 rows).  rows, cols: the valid extent from
// (r0, c0).  The buffer's 16-byte pieces are swizzled by row pair: the
// row-per-lane writes and the piece-per-lane reads are both conflict-free.
__device__ __forceinline__ void store_block_staged(__nv_bfloat16* out, int64_t ld, int r0, int c0, int rows, int cols,
                                                   const float* y, uint8_t* stg) {
  const int lane = threadIdx.x & 31;
  __syncwarp();  // the previous block's reads of the buffer are done
#pragma unroll
  for (int q = 0; q < 4; ++q)
    *reinterpret_cast<uint4*>(stg + lane * 64 + ((q ^ ((lane >> 1) & 3)) << 4)) = pack8<__nv_bfloat16>(y + 8 * q);
  __syncwarp();
  const bool vec = (ld & 7) == 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = 8 * i + (lane >> 2), q = lane & 3;
    if (r >= rows || 8 * q >= cols) continue;
    const uint4 v = *reinterpret_cast<const uint4*>(stg + r * 64 + ((q ^ ((r >> 1) & 3)) << 4));
    __nv_bfloat16* dst = out + static_cast<int64_t>(r0 + r) * ld + c0 + 8 * q;
    if (vec && 8 * q + 8 <= cols) {
      *reinterpret_cast<uint4*>(dst) = v;
    } else {
      const __nv_bfloat16* e = reinterpret_cast<const __nv_bfloat16*>(&v);
#pragma unroll
      for (int t = 0; t < 8; ++t)
        if (8 * q + t < cols) dst[t] = e[t];
    }
  }
}

// Row `row`'s 64 values v of K block `kb` into a 128 x 128 operand buffer
// (K-major, 128-byte swizzle), rounded to T; with lo, also the rounding
// remainder into the second buffer and v replaced by hi + lo.
template <typename T>
__device__ __forceinline__ void put_row(uint8_t* buf, uint8_t* buf_lo, int row, int kb, float* v, bool split) {
  uint8_t* blk = buf + kb * kKBlock;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    float hi[8], lo[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      if constexpr (std::is_same_v<T, __half>)
        hi[t] = __half2float(__float2half_rn(v[8 * q + t]));
      else
        hi[t] = __bfloat162float(__float2bfloat16_rn(v[8 * q + t]));
      lo[t] = v[8 * q + t] - hi[t];
    }
    *reinterpret_cast<uint4*>(blk + sw128_off(row, q)) = pack8<T>(hi);
    if (split) {
      *reinterpret_cast<uint4*>(buf_lo + kb * kKBlock + sw128_off(row, q)) = pack8<T>(lo);
      // the value the products see: hi + lo, each rounded to T
      float lr[8];
      const uint4 u = pack8<T>(lo);
      const T* e = reinterpret_cast<const T*>(&u);
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        if constexpr (std::is_same_v<T, __half>)
          lr[t] = __half2float(e[t]);
        else
          lr[t] = __bfloat162float(e[t]);
        v[8 * q + t] = hi[t] + lr[t];
      }
    } else {
#pragma unroll
      for (int t = 0; t < 8; ++t) v[8 * q + t] = hi[t];
    }
  }
}

// Row `row`'s 32 values v (columns 8 c4 .. 8 c4 + 31 of K block `kb`) into a
// 128 x 128 operand buffer, as put_row does for 64.
template <typename T>
__device__ __forceinline__ void put_row32(uint8_t* buf, uint8_t* buf_lo, int row, int kb, int c4, float* v,
                                          bool split) {
  uint8_t* blk = buf + kb * kKBlock;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float hi[8], lo[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      if constexpr (std::is_same_v<T, __half>)
        hi[t] = __half2float(__float2half_rn(v[8 * q + t]));
      else
        hi[t] = __bfloat162float(__float2bfloat16_rn(v[8 * q + t]));
      lo[t] = v[8 * q + t] - hi[t];
    }
    *reinterpret_cast<uint4*>(blk + sw128_off(row, c4 + q)) = pack8<T>(hi);
    if (split) {
      const uint4 u = pack8<T>(lo);
      *reinterpret_cast<uint4*>(buf_lo + kb * kKBlock + sw128_off(row, c4 + q)) = u;
      const T* e = reinterpret_cast<const T*>(&u);
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        float lr;
        if constexpr (std::is_same_v<T, __half>)
          lr = __half2float(e[t]);
        else
          lr = __bfloat162float(e[t]);
        v[8 * q + t] = hi[t] + lr;
      }
    } else {
#pragma unroll
      for (int t = 0; t < 8; ++t) v[8 * q + t] = hi[t];
    }
  }
}

__global__ void __launch_bounds__(kThreads, 1) small_kernel(const __grid_constant__ SmParams p) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* base_ptr = smem_raw + (base - raw);
  // this epilogue warp's output staging block (after the buffers and the tail)
  uint8_t* stg = base_ptr + kRing + 2 * kOpBuf + kTail + 2048 * ((threadIdx.x >> 5) >= 2 ? (threadIdx.x >> 5) - 2 : 0);
  const uint32_t ring = base;
  uint8_t* dhi = base_ptr + kRing;
  uint8_t* dlo = dhi + kOpBuf;
  const uint32_t dhi_s = base + kRing, dlo_s = dhi_s + kOpBuf;
  const uint32_t bar0 = base + kRing + 2 * kOpBuf;
  auto bar = [&](int i) { return bar0 + 8u * static_cast<uint32_t>(i); };
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(base_ptr + kRing + 2 * kOpBuf + 8 * kNumBars);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  float2* red = reinterpret_cast<float2*>(tmem_slot + 2);  // 8 epilogue warps' partial sums
  double* wco = reinterpret_cast<double*>(red + 8);         // w_0 .. w_L, then c_0 = 1 + sum w at [31]
  float* fsc = reinterpret_cast<float*>(wco + 32);          // 1/o and 1/sqrt(o), from one thread

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int mi = p.idx ? p.idx[blockIdx.x] : p.first + static_cast<int>(blockIdx.x);
  const SmProblem& pr = p.probs[mi];
  const int L = p.L;
  const int h = pr.h, w = pr.w;
  const int n_kb = (w + 63) / 64;               // K blocks of the Gram
  const int n_nt = (w + 255) / 256;             // 256-column tiles of the product
  const unsigned long long tmo = p.wait_ms ? p.wait_ms * 1000000ull : kWaitTimeoutNs;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kGramStages; ++s) {
      mbar_init(bar(kGFull + s), 1);
      mbar_init(bar(kGEmpty + s), 1);
    }
    for (int s = 0; s < kApplyStages; ++s) {
      mbar_init(bar(kAFull + s), 1);
      mbar_init(bar(kAEmpty + s), 1);
    }
    mbar_init(bar(kTFull), 1);
    mbar_init(bar(kDReady), 8);
    mbar_init(bar(kDReady1), 8);
    mbar_init(bar(kPReady), 8);
    mbar_init(bar(kGDone), 1);
    for (int a = 0; a < 2; ++a) {
      mbar_init(bar(kT2Full + a), 1);
      mbar_init(bar(kT2Empty + a), 8);
    }
    mbar_init(bar(kDrain), 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc<1>(smem_u32(tmem_slot), 512);
    tmem_relinquish<1>();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  MatScalars* sc = p.scal + mi;

  if (warp == 0) {
    if (lane == 0) {
      // ------------------------------------------------ TMA producer
      tmap_acquire(&pr.mapG);
      tmap_acquire(&pr.mapY);
      bool ok = true;
      int filled = 0, afilled = 0;
      for (int kb = 0; kb < n_kb && ok; ++kb) {
        const int s = kb % kGramStages;
        if (!mbar_wait(bar(kGEmpty + s), ((kb / kGramStages) & 1) ^ 1u, abort_flag, tmo)) {
          ok = false;
          break;
        }
        const uint32_t fb = bar(kGFull + s);
        mbar_arrive_expect_tx(fb, kKBlock);
        const uint32_t dst = ring + s * kKBlock;
        if (!pr.trans) {
          tma_load_2d(dst, &pr.mapG, fb, 64 * kb, 0);  // A = M: 128 rows x 64 K
        } else {
          tma_load_2d(dst, &pr.mapG, fb, 0, 64 * kb);  // A = M^T: two 64-wide MN chunks
          tma_load_2d(dst + 8192, &pr.mapG, fb, 64, 64 * kb);
        }
        ++filled;
      }
      // the product's stages overlay the Gram's: wait until its products have read them
      if (ok && !mbar_wait(bar(kGDone), 0, abort_flag, tmo)) ok = false;
      for (int t = 0; ok && t < 2 * n_nt; ++t) {
        const int nt = t >> 1, kb = t & 1;
        const int s = t % kApplyStages;
        if (!mbar_wait(bar(kAEmpty + s), ((t / kApplyStages) & 1) ^ 1u, abort_flag, tmo)) {
          ok = false;
          break;
        }
        const uint32_t fb = bar(kAFull + s);
        mbar_arrive_expect_tx(fb, kApplyStage);
        const uint32_t dst = ring + s * kApplyStage;
        if (!pr.trans) {
          // B(n, k) = A(k, n) = M(k, n): four 64-wide MN chunks of the tile
#pragma unroll
          for (int j = 0; j < 4; ++j) tma_load_2d(dst + 8192 * j, &pr.mapY, fb, 256 * nt + 64 * j, 64 * kb);
        } else {
          // B(n, k) = M(n, k): 256 K-major rows
          tma_load_2d(dst, &pr.mapY, fb, 64 * kb, 256 * nt);
        }
        ++afilled;
      }
      if (!ok) {
        atomicOr(&sc->status, kDevTimeout);
        // let the Gram copies already issued land before the CTA exits
        for (int s = 0; s < kGramStages && s < filled; ++s) {
          const int last = s + ((filled - 1 - s) / kGramStages) * kGramStages;
          mbar_wait_bounded(bar(kGFull + s), (last / kGramStages) & 1, tmo);
        }
        for (int s = 0; s < kApplyStages && s < afilled; ++s) {
          const int last = s + ((afilled - 1 - s) / kApplyStages) * kApplyStages;
          mbar_wait_bounded(bar(kAFull + s), (last / kApplyStages) & 1, tmo);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ------------------------------------------------ MMA issuer
      bool ok = true;
      const uint32_t acc = tmem_base;  // columns [0, 128): T_0, then each D_l^2
      // Gram: A and B are the same 128 x 64 tile (T_0 = A A^T)
      const uint32_t id_g = idesc_f16(1u, 128, 128, pr.trans ? 1u : 0u, pr.trans ? 1u : 0u);
      for (int kb = 0; kb < n_kb && ok; ++kb) {
        const int s = kb % kGramStages;
        if (!mbar_wait(bar(kGFull + s), (kb / kGramStages) & 1, abort_flag, tmo)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t sa = ring + s * kKBlock;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const uint64_t d = pr.trans ? sdesc_sw128(sa + k * 2048, 8192, 1024) : sdesc_sw128(sa + k * 32, 16, 1024);
          umma_f16<1>(acc, d, d, id_g, (kb | k) != 0 ? 1u : 0u);
        }
        umma_commit<1>(bar(kGEmpty + s));
      }
      if (ok) {
        umma_commit<1>(bar(kTFull));
        umma_commit<1>(bar(kGDone));
      }
      // squarings: D_l D_l from the FP16 operand buffers (D symmetric: B = A)
      const uint32_t id_s = idesc_f16(0u, 128, 128, 0u, 0u);
      // Squaring j accumulates in TMEM columns 128 ((j - 1) & 1) .. + 127, so
      // that its K block 0 products can start while the epilogue still turns
      // the other accumulator's K block 1 columns into the operand.
      for (int j = 1; j <= L - 1 && ok; ++j) {
        const uint32_t accj = tmem_base + 128u * static_cast<uint32_t>((j - 1) & 1);
        const bool split = j <= p.k_split;
        const int np = split ? 3 : 1;
        int first = 1;
#pragma unroll 1
        for (int kb = 0; kb < 2; ++kb) {
          if (!mbar_wait(bar(kb ? kDReady1 : kDReady), (j - 1) & 1, abort_flag, tmo)) {
            ok = false;
            break;
          }
          tc_fence_after();
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            for (int q = 0; q < np; ++q) {
              // hi hi, hi lo, lo hi
              const uint32_t sa = (q == 2 ? dlo_s : dhi_s) + kb * kKBlock + k * 32;
              const uint32_t sb = (q == 1 ? dlo_s : dhi_s) + kb * kKBlock + k * 32;
              umma_f16<1>(accj, sdesc_sw128(sa, 16, 1024), sdesc_sw128(sb, 16, 1024), id_s, first ? 0u : 1u);
              first = 0;
            }
          }
        }
        if (!ok) break;
        umma_commit<1>(bar(kTFull));
      }
      // the product Y = P A: P hi (+ lo) as the A operand, A's columns as B
      if (ok && !mbar_wait(bar(kPReady), 0, abort_flag, tmo)) ok = false;
      if (ok) tc_fence_after();
      const uint32_t id_y = idesc_f16(1u, 128, 256, 0u, pr.trans ? 0u : 1u);
      const int np = p.p_split ? 2 : 1;
      for (int nt = 0; nt < n_nt && ok; ++nt) {
        const int b = nt & 1;
        if (!mbar_wait(bar(kT2Empty + b), ((nt >> 1) & 1) ^ 1u, abort_flag, tmo)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d_t = tmem_base + static_cast<uint32_t>(256 * b);
        for (int kb = 0; kb < 2 && ok; ++kb) {
          const int t = 2 * nt + kb;
          const int s = t % kApplyStages;
          if (!mbar_wait(bar(kAFull + s), (t / kApplyStages) & 1, abort_flag, tmo)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sb = ring + s * kApplyStage;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const uint64_t bd = pr.trans ? sdesc_sw128(sb + k * 32, 16, 1024) : sdesc_sw128(sb + k * 2048, 8192, 1024);
            for (int q = 0; q < np; ++q) {
              const uint32_t sa = (q ? dlo_s : dhi_s) + kb * kKBlock + k * 32;
              umma_f16<1>(d_t, sdesc_sw128(sa, 16, 1024), bd, id_y, (kb | k | q) != 0 ? 1u : 0u);
            }
          }
          umma_commit<1>(bar(kAEmpty + s));
        }
        if (ok) umma_commit<1>(bar(kT2Full + b));
      }
      if (!ok) atomicOr(&sc->status, kDevTimeout);
      umma_commit<1>(bar(kDrain));
      mbar_wait_bounded(bar(kDrain), 0, tmo);
    }
  } else {
    // -------------------------------------------------- epilogue (warps 2..9)
    const int q = warp & 3;               // TMEM lane quadrant: rows 32 q .. 32 q + 31
    // columns 32 half .. 32 half + 31 of each K block (the K block 0 ones first)
    const int half = (warp - 2) >> 2;
    const int row = 32 * q + lane;
    auto col_of = [&](int t) { return (t < 32 ? 0 : 32) + 32 * half + t; };  // column of d[t]
    const uint32_t trow = tmem_base + (static_cast<uint32_t>(32 * q) << 16);
    auto wait_bar = [&](uint32_t b, uint32_t parity) {
      int ok = 0;
      if (lane == 0) ok = mbar_wait(b, parity, abort_flag, tmo) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (ok) tc_fence_after();
      return ok != 0;
    };
    // this thread's 64 columns (32 of each K block) of the 128 starting at `base`
    auto load_cols = [&](uint32_t base, float* v) {
      uint32_t u[32];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        IFNSO_TMEM_LD32(trow + base + 64 * c + 32 * half, u);
        IFNSO_TMEM_WAIT_LD(u);
#pragma unroll
        for (int t = 0; t < 32; ++t) v[32 * c + t] = __uint_as_float(u[t]);
      }
    };
    // TMEM: the squarings' two accumulators in columns 0..255, P (FP32) in
    // 256..383 (this thread's row, its 64 columns)
    const uint32_t tp = trow + 256 + 32 * half;
    auto p_store = [&](const float* v) {
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        uint32_t u[32];
#pragma unroll
        for (int t = 0; t < 32; ++t) u[t] = __float_as_uint(v[32 * c + t]);
        IFNSO_TMEM_ST32(tp + 64 * c, u);
      }
      tmem_wait_st();
    };
    float d[64];
    // the coefficients into shared memory while the Gram runs (the squaring
    // chain then reads no global memory); the barrier below publishes them
    if (warp == 2) {
      if (lane <= L) wco[lane] = coef_at(p.coef, mi, lane);
      __syncwarp();
      if (lane == 0) {
        double c = 1.0;
        for (int l = 1; l <= L; ++l) c += wco[l];
        wco[31] = c;
      }
    }
    bool ok = wait_bar(bar(kTFull), 0);
    float inv_s2 = 0.f, inv_s = 0.f;
    double c0 = 1.0;
    {
      float ss = 0.f, tr = 0.f;
      if (ok) {
        load_cols(0, d);
#pragma unroll
        for (int t = 0; t < 64; ++t) {
          ss = fmaf(d[t], d[t], ss);
          if (col_of(t) == row) tr += d[t];
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        ss += __shfl_xor_sync(0xffffffffu, ss, o);
        tr += __shfl_xor_sync(0xffffffffu, tr, o);
      }
      if (lane == 0) red[warp - 2] = make_float2(ss, tr);
      // every epilogue warp reaches this barrier, whether or not its wait succeeded
      asm volatile("bar.sync 1, 256;" ::: "memory");
    }
    // the FP64 scalars in one thread (the FP64 pipe is narrow: 256 threads
    // repeating the square roots and divisions took microseconds), then shared
    if (warp == 2 && lane == 0) {
      float i2 = 0.f, i1 = 0.f;
      if (ok) {
        double o2 = 0.0, trace = 0.0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          o2 += static_cast<double>(red[k].x);
          trace += static_cast<double>(red[k].y);
        }
        const double s2 = p.frob ? trace : sqrt(o2);
        const double c = wco[31];
        const bool fin = isfinite(s2) && isfinite(c);
        const bool pos = fin && s2 > 0.0;
        i2 = pos ? static_cast<float>(1.0 / s2) : 0.f;
        i1 = pos ? static_cast<float>(1.0 / sqrt(s2)) : 0.f;
        sc->o2 = o2;
        sc->trace = trace;
        sc->s2 = s2;
        sc->c0 = c;
        sc->inv_s2 = i2;
        sc->inv_s = i1;
        atomicOr(&sc->status, (!fin ? kDevNonFinite : 0) | ((fin && s2 == 0.0) ? kDevZero : 0));
      }
      fsc[0] = i2;
      fsc[1] = i1;
    }
    asm volatile("bar.sync 1, 256;" ::: "memory");  // reached by every epilogue warp
    if (ok) {
      inv_s2 = fsc[0];
      inv_s = fsc[1];
      c0 = wco[31];
      // D_1 = T_0 / o as the first squaring's operand (hi + lo when it is split)
#pragma unroll
      for (int t = 0; t < 64; ++t) d[t] *= inv_s2;
      tc_fence_before();  // (T_0 read: squaring 1 accumulates over it)
      if (L >= 2) {
#pragma unroll
        for (int kb = 0; kb < 2; ++kb) {
          put_row32<__half>(dhi, dlo, row, kb, 4 * half, d + 32 * kb, 1 <= p.k_split);
          fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) mbar_arrive(bar(kb ? kDReady1 : kDReady));
        }
      }
      const float c0f = static_cast<float>(c0);
      const float w1 = static_cast<float>(wco[1]);
      {
        float pv[64];
#pragma unroll
        for (int t = 0; t < 64; ++t) pv[t] = fmaf(-w1, d[t], (col_of(t) == row) ? c0f : 0.f);
        p_store(pv);
      }
    }
    for (int j = 1; j <= L - 1 && ok; ++j) {
      if (!(ok = wait_bar(bar(kTFull), j & 1))) break;
      const float wn = static_cast<float>(wco[j + 1]);
      const uint32_t accj = trow + 128u * static_cast<uint32_t>((j - 1) & 1);
      // K block 0's columns first: the next squaring's first products start on them
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        uint32_t u[32], pu[32];
        IFNSO_TMEM_LD32(accj + 64 * c + 32 * half, u);
        IFNSO_TMEM_LD32(tp + 64 * c, pu);
        IFNSO_TMEM_WAIT_LD(u);
        IFNSO_TMEM_WAIT_LD(pu);
#pragma unroll
        for (int t = 0; t < 32; ++t) {
          const float dn = 2.0f * d[32 * c + t] - __uint_as_float(u[t]);  // D_{j+1} = 2 D_j - D_j^2
          d[32 * c + t] = dn;
          pu[t] = __float_as_uint(fmaf(-wn, dn, __uint_as_float(pu[t])));  // P -= w_{j+1} D_{j+1}
        }
        IFNSO_TMEM_ST32(tp + 64 * c, pu);
        if (j < L - 1) {
          tc_fence_before();
          put_row32<__half>(dhi, dlo, row, c, 4 * half, d + 32 * c, j + 1 <= p.k_split);
          fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) mbar_arrive(bar(c ? kDReady1 : kDReady));
        }
      }
      tmem_wait_st();
      tc_fence_before();
    }
    if (ok) {
      // P as BF16 hi (+ lo): the A operand of the product (P is symmetric)
      load_cols(256, d);
      tc_fence_before();  // the product's accumulator 1 overwrites these TMEM columns
#pragma unroll
      for (int kb = 0; kb < 2; ++kb) put_row32<__nv_bfloat16>(dhi, dlo, row, kb, 4 * half, d + 32 * kb, p.p_split != 0);
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(kPReady));
    }
    // Y = P A / sqrt(o): this warp's rows, 128 of each tile's 256 columns
    __nv_bfloat16* out = static_cast<__nv_bfloat16*>(pr.out);
    for (int nt = 0; nt < n_nt && ok; ++nt) {
      const int b = nt & 1;
      if (!(ok = wait_bar(bar(kT2Full + b), (nt >> 1) & 1))) break;
#pragma unroll 1
      for (int c = 0; c < 4; ++c) {
        const int col = 256 * nt + 128 * half + 32 * c;  // first output column (of A's w)
        uint32_t u[32];
        __syncwarp();
        IFNSO_TMEM_LD32(trow + static_cast<uint32_t>(256 * b + 128 * half + 32 * c), u);
        IFNSO_TMEM_WAIT_LD(u);
        if (col >= w) continue;  // (warp-uniform; the loop head reconverges the warp before the next load)
        float y[32];
#pragma unroll
        for (int t = 0; t < 32; ++t) y[t] = __uint_as_float(u[t]) * inv_s;
        if (!pr.trans) {
          store_block_staged(out, pr.ld_out, 32 * q, col, h - 32 * q, w - col, y, stg);
        } else if (row < h) {
          // M is tall: Y^T, element (row, col + t) goes to out[col + t][row]
          // (consecutive lanes write consecutive elements)
#pragma unroll
          for (int t = 0; t < 32; ++t)
            if (col + t < w) out[static_cast<int64_t>(col + t) * pr.ld_out + row] = __float2bfloat16_rn(y[t]);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(kT2Empty + b));
    }
    if (!ok && lane == 0) atomicOr(&sc->status, kDevTimeout);
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc<1>(tmem_base, 512);
  }
}


// ------------------------------------------------------------------------
// The Newton-Schulz baseline (Sec. 1, Eqs. one_iteration_matrix and
// iteration_jordan) on chip for h <= 128, one CTA per matrix: per step
//   S = X X^T (tcgen05, X streamed over K = w), B = b S + c S^2 (quintic;
//   the cubic iteration takes B = b S), X <- a X + B X (X streamed again in
//   256-column tiles).
// X_0 = A / ||A||_F with ||A||_F^2 = tr(A A^T) from the first Gram.  The
// product's epilogue reads X from the shared-memory stages that hold its B
// operand and writes X_{k+1} back into them; the producer, before it
// refills those stages, moves them with TMA stores to a workspace buffer
// (M's layout) that the next step streams in.  The last step writes Y in M's
// shape.
enum NsBar {
  nGFull = 0,
  nGEmpty = nGFull + kGramStages,
  nAFull = nGEmpty + kGramStages,
  nTFull = nAFull + kApplyStages,   // S, then S^2, in TMEM columns 0..127
  nSReady,                          // S (BF16) written (8 epilogue warps)
  nBReady,                          // B (BF16) written (8 epilogue warps)
  nGDone,                           // this step's Gram products have read their stages
  nT2Full,
  nT2Empty = nT2Full + 2,
  nXReady = nT2Empty + 2,           // X_{k+1} stored in global memory (the producer)
  nTileDone,                        // the 8 epilogue warps are done with a product tile's stages
  nTileDone1 = nTileDone + 1,       // (even and odd tiles)
  nDrain,
  nNumBars
};
static_assert(nNumBars * 8 + 8 + 8 * 8 + 8 <= kTail, "barriers, TMEM slot, abort flag, 8 partial sums, 2 scalars");

// Byte offset of X(i, n) (M tall: the tile's rows are n) in a 256-column
// B-operand tile held as two stages of 256 K-major rows (128-byte swizzle).
__device__ __forceinline__ uint32_t xstage_off_tall(int i, int nl) {
  const int kb = i >> 6, k = i & 63;
  return static_cast<uint32_t>(kb * kApplyStage + (nl >> 3) * 1024 + (nl & 7) * 128 +
                               ((((k >> 3) ^ (nl & 7))) << 4) + (k & 7) * 2);
}

__global__ void __launch_bounds__(kThreads, 1) small_ns_kernel(const __grid_constant__ SmNsParams p) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* base_ptr = smem_raw + (base - raw);
  // this epilogue warp's output staging block (after the buffers and the tail)
  uint8_t* stg = base_ptr + kRing + 2 * kOpBuf + kTail + 2048 * ((threadIdx.x >> 5) >= 2 ? (threadIdx.x >> 5) - 2 : 0);
  const uint32_t ring = base;
  uint8_t* sbuf = base_ptr + kRing;  // S (BF16 operand)
  uint8_t* bbuf = sbuf + kOpBuf;     // B (BF16 operand)
  const uint32_t sbuf_s = base + kRing, bbuf_s = sbuf_s + kOpBuf;
  const uint32_t bar0 = base + kRing + 2 * kOpBuf;
  auto bar = [&](int i) { return bar0 + 8u * static_cast<uint32_t>(i); };
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(base_ptr + kRing + 2 * kOpBuf + 8 * nNumBars);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  float2* red = reinterpret_cast<float2*>(tmem_slot + 2);
  float* fsc = reinterpret_cast<float*>(red + 8);  // 1/||A||_F^2 and 1/||A||_F, from one thread

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int mi = p.first + static_cast<int>(blockIdx.x);
  const SmNsProblem& pr = p.probs[mi];
  const int h = pr.h, w = pr.w, steps = p.steps;
  const bool quintic = p.degree == 5;
  const int n_kb = (w + 63) / 64;
  const int n_nt = (w + 255) / 256;
  const unsigned long long tmo = p.wait_ms ? p.wait_ms * 1000000ull : kWaitTimeoutNs;
  auto src_of = [&](int s) { return s == 0 ? 0 : 1 + ((s - 1) & 1); };  // A, X0, X1
  auto dst_of = [&](int s) { return 1 + (s & 1); };

  if (threadIdx.x == 0) {
    for (int s = 0; s < kGramStages; ++s) {
      mbar_init(bar(nGFull + s), 1);
      mbar_init(bar(nGEmpty + s), 1);
    }
    for (int s = 0; s < kApplyStages; ++s) {
      mbar_init(bar(nAFull + s), 1);
    }
    mbar_init(bar(nTFull), 1);
    mbar_init(bar(nSReady), 8);
    mbar_init(bar(nBReady), 8);
    mbar_init(bar(nGDone), 1);
    for (int a = 0; a < 2; ++a) {
      mbar_init(bar(nT2Full + a), 1);
      mbar_init(bar(nT2Empty + a), 8);
    }
    mbar_init(bar(nXReady), 1);
    mbar_init(bar(nTileDone), 8);
    mbar_init(bar(nTileDone1), 8);
    mbar_init(bar(nDrain), 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc<1>(smem_u32(tmem_slot), 512);
    tmem_relinquish<1>();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  MatScalars* sc = p.scal + mi;

  if (warp == 0) {
    if (lane == 0) {
      // ------------------------------------------------ TMA producer
      for (int m = 0; m < 3; ++m) {
        tmap_acquire(&pr.mapG[m]);
        tmap_acquire(&pr.mapY[m]);
      }
      bool ok = true;
      int g = 0, t = 0, tg = 0;  // Gram and product loads, product tiles, so far (over all steps)
      // the 8 epilogue warps are done with product tile x (its stages hold X_{k+1})
      auto tile_done = [&](int x) { return mbar_wait(bar(nTileDone + (x & 1)), (x >> 1) & 1, abort_flag, tmo); };
      // TMA stores of tile x (tile nt of its step) to X buffer di: only boxes
      // that start inside X (the rest of a box is clipped)
      auto store_tile = [&](int x, int nt, int di) {
        const uint32_t src = ring + 2u * static_cast<uint32_t>(x & 1) * kApplyStage;
        for (int kb = 0; kb < 2 && 64 * kb < h; ++kb) {
          if (!pr.trans) {
            for (int j = 0; j < 4 && 256 * nt + 64 * j < w; ++j)
              tma_store_2d(&pr.mapY[di], src + kb * kApplyStage + 8192 * j, 256 * nt + 64 * j, 64 * kb);
          } else {
            tma_store_2d(&pr.mapY[di], src + kb * kApplyStage, 64 * kb, 256 * nt);
          }
        }
        bulk_commit();
      };
      for (int st = 0; st < steps && ok; ++st) {
        const int si = src_of(st), di = dst_of(st);
        const bool last = st == steps - 1;
        // (the previous step's tiles were stored and their stages read below)
        for (int kb = 0; kb < n_kb && ok; ++kb, ++g) {
          const int s = g % kGramStages;
          if (!mbar_wait(bar(nGEmpty + s), ((g / kGramStages) & 1) ^ 1u, abort_flag, tmo)) {
            ok = false;
            break;
          }
          const uint32_t fb = bar(nGFull + s);
          mbar_arrive_expect_tx(fb, kKBlock);
          const uint32_t dst = ring + s * kKBlock;
          if (!pr.trans) {
            tma_load_2d(dst, &pr.mapG[si], fb, 64 * kb, 0);
          } else {
            tma_load_2d(dst, &pr.mapG[si], fb, 0, 64 * kb);
            tma_load_2d(dst + 8192, &pr.mapG[si], fb, 64, 64 * kb);
          }
        }
        if (ok && !mbar_wait(bar(nGDone), st & 1, abort_flag, tmo)) ok = false;
        // product tiles: tile x takes stages 2 (x & 1) and 2 (x & 1) + 1; before
        // they are refilled, the tile two before has been written back by the
        // epilogue, stored to X_{k+1} and read by the stores
        const int tg0 = tg;
        for (int nt = 0; ok && nt < n_nt; ++nt) {
          const int x = tg0 + nt;
          if (nt >= 2) {
            if (!tile_done(x - 2)) {
              ok = false;
              break;
            }
            if (!last) {
              store_tile(x - 2, nt - 2, di);
              bulk_wait_read();
            }
          }
          for (int kb = 0; kb < 2; ++kb, ++t) {
            const int s = t % kApplyStages;  // = 2 (x & 1) + kb
            const uint32_t fb = bar(nAFull + s);
            mbar_arrive_expect_tx(fb, kApplyStage);
            const uint32_t dst = ring + s * kApplyStage;
            if (!pr.trans) {
#pragma unroll
              for (int j = 0; j < 4; ++j) tma_load_2d(dst + 8192 * j, &pr.mapY[si], fb, 256 * nt + 64 * j, 64 * kb);
            } else {
              tma_load_2d(dst, &pr.mapY[si], fb, 64 * kb, 256 * nt);
            }
          }
        }
        if (ok && !last) {
          // the step's last tiles; then X_{k+1} is in global memory for the next step
          for (int nt = n_nt > 2 ? n_nt - 2 : 0; ok && nt < n_nt; ++nt) {
            if (!tile_done(tg0 + nt)) {
              ok = false;
              break;
            }
            store_tile(tg0 + nt, nt, di);
          }
          if (ok) {
            bulk_wait_all();
            fence_proxy_async_global();
            mbar_arrive(bar(nXReady));
          }
        }
        tg = tg0 + n_nt;
      }
      if (!ok) {
        atomicOr(&sc->status, kDevTimeout);
        // let the copies issued last land: every ring stage's latest phase
        for (int s = 0; s < kGramStages && s < g; ++s) {
          const int last = s + ((g - 1 - s) / kGramStages) * kGramStages;
          mbar_wait_bounded(bar(nGFull + s), (last / kGramStages) & 1, tmo);
        }
        for (int s = 0; s < kApplyStages && s < t; ++s) {
          const int last = s + ((t - 1 - s) / kApplyStages) * kApplyStages;
          mbar_wait_bounded(bar(nAFull + s), (last / kApplyStages) & 1, tmo);
        }
      }
      bulk_wait_all();  // no store in flight when the CTA exits
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ------------------------------------------------ MMA issuer
      bool ok = true;
      const uint32_t acc = tmem_base;
      const uint32_t id_g = idesc_f16(1u, 128, 128, pr.trans ? 1u : 0u, pr.trans ? 1u : 0u);
      const uint32_t id_s = idesc_f16(1u, 128, 128, 0u, 0u);
      const uint32_t id_y = idesc_f16(1u, 128, 256, 0u, pr.trans ? 0u : 1u);
      int g = 0, t = 0, ntg = 0;
      for (int st = 0; st < steps && ok; ++st) {
        if (st > 0) {
          // the previous step's epilogue has drained every accumulator
          if (!mbar_wait(bar(nXReady), (st - 1) & 1, abort_flag, tmo)) {
            ok = false;
            break;
          }
          tc_fence_after();
        }
        for (int kb = 0; kb < n_kb && ok; ++kb, ++g) {
          const int s = g % kGramStages;
          if (!mbar_wait(bar(nGFull + s), (g / kGramStages) & 1, abort_flag, tmo)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = ring + s * kKBlock;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const uint64_t d = pr.trans ? sdesc_sw128(sa + k * 2048, 8192, 1024) : sdesc_sw128(sa + k * 32, 16, 1024);
            umma_f16<1>(acc, d, d, id_g, (kb | k) != 0 ? 1u : 0u);
          }
          umma_commit<1>(bar(nGEmpty + s));
        }
        if (!ok) break;
        umma_commit<1>(bar(nTFull));
        umma_commit<1>(bar(nGDone));
        if (quintic) {
          if (!mbar_wait(bar(nSReady), st & 1, abort_flag, tmo)) {
            ok = false;
            break;
          }
          tc_fence_after();
          for (int kb = 0; kb < 2; ++kb)
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const uint64_t d = sdesc_sw128(sbuf_s + kb * kKBlock + k * 32, 16, 1024);
              umma_f16<1>(acc, d, d, id_s, (kb | k) != 0 ? 1u : 0u);
            }
          umma_commit<1>(bar(nTFull));
        }
        if (!mbar_wait(bar(nBReady), st & 1, abort_flag, tmo)) {
          ok = false;
          break;
        }
        tc_fence_after();
        for (int nt = 0; nt < n_nt && ok; ++nt, ++ntg) {
          const int b = ntg & 1;
          if (!mbar_wait(bar(nT2Empty + b), ((ntg >> 1) & 1) ^ 1u, abort_flag, tmo)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d_t = tmem_base + static_cast<uint32_t>(256 * b);
          for (int kb = 0; kb < 2 && ok; ++kb, ++t) {
            const int s = t % kApplyStages;
            if (!mbar_wait(bar(nAFull + s), (t / kApplyStages) & 1, abort_flag, tmo)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t sb = ring + s * kApplyStage;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const uint64_t bd = pr.trans ? sdesc_sw128(sb + k * 32, 16, 1024) : sdesc_sw128(sb + k * 2048, 8192, 1024);
              const uint64_t ad = sdesc_sw128(bbuf_s + kb * kKBlock + k * 32, 16, 1024);
              umma_f16<1>(d_t, ad, bd, id_y, (kb | k) != 0 ? 1u : 0u);
            }
            // (the stage is released by the epilogue, which reads X from it)
          }
          if (ok) umma_commit<1>(bar(nT2Full + b));
        }
      }
      if (!ok) atomicOr(&sc->status, kDevTimeout);
      umma_commit<1>(bar(nDrain));
      mbar_wait_bounded(bar(nDrain), 0, tmo);
    }
  } else {
    // -------------------------------------------------- epilogue (warps 2..9)
    const int q = warp & 3;
    const int half = (warp - 2) >> 2;
    const int row = 32 * q + lane;
    const uint32_t trow = tmem_base + (static_cast<uint32_t>(32 * q) << 16);
    const bool leader = warp == 2 && lane == 0;
    auto wait_bar = [&](uint32_t b, uint32_t parity) {
      int ok = 0;
      if (lane == 0) ok = mbar_wait(b, parity, abort_flag, tmo) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (ok) tc_fence_after();
      return ok != 0;
    };
    auto load64 = [&](uint32_t col, float* v) {
      uint32_t u[32];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        IFNSO_TMEM_LD32(trow + col + 32 * c, u);
        IFNSO_TMEM_WAIT_LD(u);
#pragma unroll
        for (int t = 0; t < 32; ++t) v[32 * c + t] = __uint_as_float(u[t]);
      }
    };
    float d[64];
    float inv_s2 = 0.f, inv_s = 0.f;
    bool ok = true;
    int tf = 0, ntg = 0, t = 0;
    __nv_bfloat16* out = static_cast<__nv_bfloat16*>(pr.out);
    for (int st = 0; st < steps && ok; ++st) {
      const bool last = st == steps - 1;
      // S = X X^T (step 0: A A^T / ||A||_F^2)
      ok = wait_bar(bar(nTFull), (tf++) & 1);
      if (st == 0) {
        float tr = 0.f;
        if (ok) {
          load64(64 * half, d);
#pragma unroll
          for (int k = 0; k < 64; ++k)
            if (64 * half + k == row) tr += d[k];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
        if (lane == 0) red[warp - 2] = make_float2(0.f, tr);
        asm volatile("bar.sync 1, 256;" ::: "memory");  // reached by every epilogue warp
        // the FP64 scalars in one thread, then shared
        if (leader) {
          float i2 = 0.f, i1 = 0.f;
          if (ok) {
            double trace = 0.0;
#pragma unroll
            for (int k = 0; k < 8; ++k) trace += static_cast<double>(red[k].y);
            const bool fin = isfinite(trace);
            const bool pos = fin && trace > 0.0;
            i2 = pos ? static_cast<float>(1.0 / trace) : 0.f;
            i1 = pos ? static_cast<float>(1.0 / sqrt(trace)) : 0.f;
            sc->trace = trace;
            sc->s2 = trace;
            sc->inv_s2 = i2;
            sc->inv_s = i1;
            atomicOr(&sc->status, (!fin ? kDevNonFinite : 0) | ((fin && trace == 0.0) ? kDevZero : 0));
          }
          fsc[0] = i2;
          fsc[1] = i1;
        }
        asm volatile("bar.sync 1, 256;" ::: "memory");  // reached by every epilogue warp
        inv_s2 = fsc[0];
        inv_s = fsc[1];
#pragma unroll
        for (int k = 0; k < 64; ++k) d[k] *= inv_s2;
      } else if (ok) {
        load64(64 * half, d);
      }
      if (!ok) break;
      put_row<__nv_bfloat16>(sbuf, nullptr, row, half, d, false);  // d becomes the BF16 S
      fence_proxy_async_smem();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(nSReady));
      // B = b S + c S^2 (or b S)
      if (quintic) {
        if (!(ok = wait_bar(bar(nTFull), (tf++) & 1))) break;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          uint32_t u[32];
          IFNSO_TMEM_LD32(trow + 64 * half + 32 * c, u);
          IFNSO_TMEM_WAIT_LD(u);
#pragma unroll
          for (int k = 0; k < 32; ++k) d[32 * c + k] = fmaf(p.c, __uint_as_float(u[k]), p.b * d[32 * c + k]);
        }
        tc_fence_before();
      } else {
#pragma unroll
        for (int k = 0; k < 64; ++k) d[k] *= p.b;
      }
      put_row<__nv_bfloat16>(bbuf, nullptr, row, half, d, false);
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(nBReady));
      // X <- a X + B X, tile by tile; X comes from the stages of the product's B operand
      const float sx = st == 0 ? inv_s : 1.f;
      for (int nt = 0; nt < n_nt; ++nt, ++ntg, t += 2) {
        const int b = ntg & 1;
        if (!(ok = wait_bar(bar(nT2Full + b), (ntg >> 1) & 1))) break;
        const uint8_t* stage0 = base_ptr + (t % kApplyStages) * kApplyStage;  // the tile's two stages are adjacent
#pragma unroll 1
        for (int c = 0; c < 4; ++c) {
          const int nl = 128 * half + 32 * c;  // first column within the tile
          const int col = 256 * nt + nl;
          uint32_t u[32];
          __syncwarp();
          IFNSO_TMEM_LD32(trow + static_cast<uint32_t>(256 * b + nl), u);
          IFNSO_TMEM_WAIT_LD(u);
          float y[32];
          // X(row, col + k): M wide, four 16-byte pieces of the row (one 128-byte
          // swizzled row of a 64 x 64 chunk; eight consecutive rows hit eight
          // distinct 16-byte bank groups); M tall, one value per 128-byte row
          uint8_t* xrow = nullptr;
          if (!pr.trans) {
            xrow = const_cast<uint8_t*>(stage0) + (row >> 6) * kApplyStage + 8192 * (nl >> 6) + (row & 63) * 128;
#pragma unroll
            for (int v = 0; v < 4; ++v) {
              const uint4 q8 = *reinterpret_cast<const uint4*>(xrow + (((((nl & 63) >> 3) + v) ^ (row & 7)) << 4));
              const __nv_bfloat162* e = reinterpret_cast<const __nv_bfloat162*>(&q8);
#pragma unroll
              for (int t = 0; t < 4; ++t) {
                const float2 f = __bfloat1622float2(e[t]);
                y[8 * v + 2 * t] = sx * fmaf(p.a, f.x, __uint_as_float(u[8 * v + 2 * t]));
                y[8 * v + 2 * t + 1] = sx * fmaf(p.a, f.y, __uint_as_float(u[8 * v + 2 * t + 1]));
              }
            }
          } else {
#pragma unroll
            for (int k = 0; k < 32; ++k) {
              const uint32_t off = xstage_off_tall(row, nl + k);
              const float x = __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(stage0 + off));
              y[k] = sx * fmaf(p.a, x, __uint_as_float(u[k]));
            }
          }
          if (last) {
            if (col < w) {  // (warp-uniform)
              if (!pr.trans) {
                store_block_staged(out, pr.ld_out, 32 * q, col, h - 32 * q, w - col, y, stg);
              } else if (row < h) {
#pragma unroll
                for (int k = 0; k < 32; ++k)
                  if (col + k < w) out[static_cast<int64_t>(col + k) * pr.ld_out + row] = __float2bfloat16_rn(y[k]);
              }
            }
          } else {
            // X_{st+1}(row, col + k) back into the stage, where the TMA store reads it
            if (!pr.trans) {
#pragma unroll
              for (int v = 0; v < 4; ++v)
                *reinterpret_cast<uint4*>(xrow + (((((nl & 63) >> 3) + v) ^ (row & 7)) << 4)) =
                    pack8<__nv_bfloat16>(y + 8 * v);
            } else {
#pragma unroll
              for (int k = 0; k < 32; ++k)
                *reinterpret_cast<__nv_bfloat16*>(const_cast<uint8_t*>(stage0) + xstage_off_tall(row, nl + k)) =
                    __float2bfloat16_rn(y[k]);
            }
          }
        }
        tc_fence_before();
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(bar(nT2Empty + b));
          mbar_arrive(bar(nTileDone + b));  // the producer stores the stages and refills them
        }
      }
      if (!ok) break;
    }
    if (!ok && lane == 0) atomicOr(&sc->status, kDevTimeout);
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc<1>(tmem_base, 512);
  }
}

}  // namespace

cudaError_t launch_small_ns(const SmNsParams& p, int count, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(small_ns_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  small_ns_kernel<<<count, kThreads, kSmem, s>>>(p);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_small(const SmParams& p, int count, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  small_kernel<<<count, kThreads, kSmem, s>>>(p);
  count_launch();
  return cudaGetLastError();
}

}  // namespace ifnso
