// Persistent, grouped tcgen05 GEMM for the IFNSO passes and the Newton-Schulz
// baseline (sm_103a).
//
// One launch runs one pass of Algorithm 1 (Sec. 2.4) for every matrix of a
// batch: the Gram product T_0 = A A^T, one squaring T_{l+1} = T_l^2 (in the
// D basis, D_{l+1} = 2 D_l - D_l^2), or the final product Y = Y' A / sqrt(o).
// Clusters of two CTAs (one CTA per SM) walk a static list of pairs of
// 128 x 256 output tiles that share their B operand: each CTA computes one
// tile of the pair and TMA-multicasts its half of the shared B tile to both.
//
// Warp roles (320 threads):
//   warp 0      TMA producer: K blocks of 64 of every operand source into a
//               ring of shared-memory stages (128-byte swizzle).
//   warp 1      TMEM owner (512 columns = two 128 x 256 FP32 accumulators)
//               and MMA issuer: tcgen05.mma M=128, N=256, K=16, kind::f16.
//   warps 2..9  epilogue (two warps per TMEM lane quadrant, 128 columns each):
//               tcgen05.ld of the accumulator, fused elementwise math of the
//               pass, stores to global memory.
// The two accumulators let the epilogue of tile t overlap the main loop of
// tile t + 1.  Symmetric outputs (T_0, D_l, P) are computed on the upper
// 256 x 256 blocks only and stored twice (direct and mirrored).
//
// Every wait is bounded (ptx.cuh): on a timeout the CTA raises a shared
// abort flag, records IFNSO_DEV_TIMEOUT in the matrix status word, lets its
// outstanding TMA copies and MMAs land, frees TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "ptx.cuh"

namespace ifnso {

namespace {

constexpr int kEpiWarps = 8;                  // two per TMEM lane quadrant, 128 columns each
constexpr int kThreads = 64 + 32 * kEpiWarps;  // producer warp, MMA warp, epilogue warps
constexpr uint32_t kTileA = BM * BK * 2;  // 16 KB: 128 rows x 64 K of 16-bit values
constexpr uint32_t kTileB = BN * BK * 2;  // 32 KB: 256 rows x 64 K
constexpr uint32_t kTmemCols = 512;
constexpr int kStageLd = 33;                               // padded row of a transpose buffer
constexpr uint32_t kStageBytes = kEpiWarps * 32 * kStageLd * 4;  // one 32 x 33 float buffer per epilogue warp
constexpr int kDevTimeout = 4;  // IFNSO_DEV_TIMEOUT

template <int NA, int NB>
struct Cfg {
  static constexpr uint32_t stage_bytes = NA * kTileA + NB * kTileB;
  static constexpr int stages_fit = static_cast<int>((200u * 1024u) / stage_bytes);
  static constexpr int stages = stages_fit > 6 ? 6 : stages_fit;
  // tiles + 1 KB alignment slack + barriers / flags + epilogue transpose buffers
  static constexpr uint32_t smem = stages * stage_bytes + 1024 + 256 + kStageBytes;
};

// Number of products per K step: every (A source, B source) pair except
// (lo, lo): hi*hi + hi*lo + lo*hi for split operands.
template <int NA, int NB>
struct Products {
  static constexpr int n = NA * NB - ((NA == 2 && NB == 2) ? 1 : 0);
  __device__ static constexpr int a(int i) { return (NA == 2 && NB == 2) ? (i == 2 ? 1 : 0) : (NA == 2 ? i : 0); }
  __device__ static constexpr int b(int i) { return (NA == 2 && NB == 2) ? (i == 1 ? 1 : 0) : (NB == 2 ? i : 0); }
};

__device__ __forceinline__ float u2f(uint32_t u) { return __uint_as_float(u); }

__device__ __forceinline__ float warp_reduce_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ void set_timeout(MatScalars* scal, int mat) {
  atomicOr(&scal[mat].status, kDevTimeout);
}

// ---------------------------------------------------------------- epilogues

__device__ __forceinline__ void load_h32(const __half* src, float* d) {
  const uint4* s4 = reinterpret_cast<const uint4*>(src);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    uint4 u = s4[j];
    const __half2* h2 = reinterpret_cast<const __half2*>(&u);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      float2 f = __half22float2(h2[t]);
      d[8 * j + 2 * t] = f.x;
      d[8 * j + 2 * t + 1] = f.y;
    }
  }
}

__device__ __forceinline__ void load_b32(const __nv_bfloat16* src, float* d) {
  const uint4* s4 = reinterpret_cast<const uint4*>(src);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    uint4 u = s4[j];
    const __nv_bfloat162* h2 = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      float2 f = __bfloat1622float2(h2[t]);
      d[8 * j + 2 * t] = f.x;
      d[8 * j + 2 * t + 1] = f.y;
    }
  }
}

__device__ __forceinline__ void store_h32(__half* dst, const float* v) {
  uint4* d4 = reinterpret_cast<uint4*>(dst);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    uint4 u;
    __half2* h2 = reinterpret_cast<__half2*>(&u);
#pragma unroll
    for (int t = 0; t < 4; ++t) h2[t] = __floats2half2_rn(v[8 * j + 2 * t], v[8 * j + 2 * t + 1]);
    d4[j] = u;
  }
}

__device__ __forceinline__ void store_b32(__nv_bfloat16* dst, const float* v) {
  uint4* d4 = reinterpret_cast<uint4*>(dst);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    uint4 u;
    __nv_bfloat162* h2 = reinterpret_cast<__nv_bfloat162*>(&u);
#pragma unroll
    for (int t = 0; t < 4; ++t)
      h2[t] = __floats2bfloat162_rn(v[8 * j + 2 * t], v[8 * j + 2 * t + 1]);
    d4[j] = u;
  }
}

// Per-warp 32 x 32 transpose through shared memory (rows padded to 33
// floats: conflict-free in both directions).  Lane t holds v[0..31] = row
// t of a 32 x 32 block; afterwards it holds w[0..31] = column t.  Every lane
// of the warp must call it.

__device__ __forceinline__ void warp_transpose(float* st, const float* v, float* w) {
  const int lane = threadIdx.x & 31;
  __syncwarp();
#pragma unroll
  for (int j = 0; j < 32; ++j) st[lane * kStageLd + j] = v[j];
  __syncwarp();
#pragma unroll
  for (int i = 0; i < 32; ++i) w[i] = st[i * kStageLd + lane];
}

template <typename T>
__device__ __forceinline__ void store_row32(T* dst, const float* v);
template <>
__device__ __forceinline__ void store_row32<float>(float* dst, const float* v) {
  float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll
  for (int j = 0; j < 8; ++j) d4[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
}
template <>
__device__ __forceinline__ void store_row32<__half>(__half* dst, const float* v) {
  store_h32(dst, v);
}
template <>
__device__ __forceinline__ void store_row32<__nv_bfloat16>(__nv_bfloat16* dst, const float* v) {
  store_b32(dst, v);
}

// Store a 32-wide row chunk of a symmetric h_pad x h_pad result at
// (r, c0..c0+31) and, for tiles off the diagonal blocks, at (c0..c0+31, r):
// the mirrored chunk is transposed through shared memory so that every lane
// writes one contiguous 32-element row segment.  `mirror` is warp-uniform.
template <typename T>
__device__ __forceinline__ void store_sym(T* buf, int64_t ld, int r, int c0, const float* v,
                                          bool mirror, float* st) {
  store_row32<T>(buf + static_cast<int64_t>(r) * ld + c0, v);
  if (mirror) {
    float w[32];
    warp_transpose(st, v, w);
    const int lane = threadIdx.x & 31;
    store_row32<T>(buf + static_cast<int64_t>(c0 + lane) * ld + (r - lane), w);
  }
}

// Bounds-checked BF16 store of a 32-wide chunk of an output tile (row r,
// columns c0..c0+31).  With out_trans the tile is the transpose of the
// output: the chunk is transposed through shared memory and lane t writes
// output row c0 + t, columns (r - lane)..(r - lane + 31).  Warp-uniform call.
__device__ __forceinline__ void store_out_bf16(const TcProblem& pr, int r, int c0, const float* v,
                                               float* st) {
  __nv_bfloat16* out = static_cast<__nv_bfloat16*>(pr.out0);
  const bool vec_ld = (pr.ld_out & 7) == 0;
  if (!pr.out_trans) {
    if (r >= pr.rows_out) return;
    __nv_bfloat16* o = out + static_cast<int64_t>(r) * pr.ld_out + c0;
    if (c0 + 32 <= pr.cols_out && vec_ld) {
      store_b32(o, v);
    } else {
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (c0 + j < pr.cols_out) o[j] = __float2bfloat16_rn(v[j]);
    }
  } else {
    float w[32];
    warp_transpose(st, v, w);
    const int lane = threadIdx.x & 31;
    const int orow = c0 + lane, ocol = r - lane;
    if (orow >= pr.rows_out) return;
    __nv_bfloat16* o = out + static_cast<int64_t>(orow) * pr.ld_out + ocol;
    if (ocol + 32 <= pr.cols_out && vec_ld) {
      store_b32(o, w);
    } else {
#pragma unroll
      for (int i = 0; i < 32; ++i)
        if (ocol + i < pr.cols_out) o[i] = __float2bfloat16_rn(w[i]);
    }
  }
}

// Load the 32 values of the NS iterate X at the positions a chunk of the
// output tile is written to (same layout rules as store_out_bf16; zero
// outside the matrix).  Warp-uniform call.
__device__ __forceinline__ void load_x_bf16(const TcProblem& pr, int r, int c0, float* x, float* st) {
  const __nv_bfloat16* X = static_cast<const __nv_bfloat16*>(pr.aux0);
  const bool vec_ld = (pr.ld_aux & 7) == 0;
  if (!pr.out_trans) {
#pragma unroll
    for (int j = 0; j < 32; ++j) x[j] = 0.f;
    if (r >= pr.rows_out) return;
    const __nv_bfloat16* s = X + static_cast<int64_t>(r) * pr.ld_aux + c0;
    if (c0 + 32 <= pr.cols_out && vec_ld) {
      load_b32(s, x);
    } else {
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (c0 + j < pr.cols_out) x[j] = __bfloat162float(s[j]);
    }
  } else {
    // lane t reads row c0 + t of X, columns (r - lane)..+31, then the block is transposed
    const int lane = threadIdx.x & 31;
    const int xrow = c0 + lane, xcol = r - lane;
    float u[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) u[i] = 0.f;
    if (xrow < pr.rows_out) {
      const __nv_bfloat16* s = X + static_cast<int64_t>(xrow) * pr.ld_aux + xcol;
      if (xcol + 32 <= pr.cols_out && vec_ld) {
        load_b32(s, u);
      } else {
#pragma unroll
        for (int i = 0; i < 32; ++i)
          if (xcol + i < pr.cols_out) u[i] = __bfloat162float(s[i]);
      }
    }
    warp_transpose(st, u, x);
  }
}

struct EpiAcc {
  float ss;  // sum of squares (EPI_GRAM)
  float tr;  // trace contribution (EPI_GRAM)
};

template <int EPI>
__device__ __forceinline__ void epilogue_chunk(const TcParams& p, const TcProblem& pr,
                                               const WorkItem& wi, int r, int c0, float* v,
                                               EpiAcc& ea, float* st) {
  const bool mirror = (wi.flags & 1) == 0;
  if constexpr (EPI == EPI_GRAM) {
    store_sym<float>(pr.pacc, pr.ld_aux, r, c0, v, mirror, st);
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      ea.ss = fmaf(v[j], v[j], ea.ss);
      if (c0 + j == r) ea.tr += v[j];
    }
  } else if constexpr (EPI == EPI_SQR) {
    float d[32], lo[32];
    const int64_t off = static_cast<int64_t>(r) * pr.ld_aux + c0;
    load_h32(static_cast<const __half*>(pr.aux0) + off, d);
    if (p.read_lo) {
      load_h32(static_cast<const __half*>(pr.aux1) + off, lo);
#pragma unroll
      for (int j = 0; j < 32; ++j) d[j] += lo[j];
    }
    // P = (1 + sum w) I - sum_l w_l D_l is accumulated two terms at a time:
    // p_mode 1 (first squaring) writes P = c0 I - w_l D_l - w_{l+1} D_{l+1},
    // p_mode 2 subtracts w_l D_l + w_{l+1} D_{l+1}, p_mode 3 only
    // w_{l+1} D_{l+1} (last squaring after an even count), p_mode 0 leaves P.
    if (p.feat) {
      // sum of (D_1^2)_ij^2 = tr(D_1^4), a feature of the coefficient proposal
#pragma unroll
      for (int j = 0; j < 32; ++j) ea.ss = fmaf(v[j], v[j], ea.ss);
    }
    const float w = static_cast<float>(coef_at(p.coef, pr.mat, p.coef_l));
    const float wp = (p.p_mode == 1 || p.p_mode == 2 || p.p_mode == 4)
                         ? static_cast<float>(coef_at(p.coef, pr.mat, p.coef_l - 1)) : 0.f;
    float* P = pr.pacc + off;
    float pv[32];
    if (p.p_mode == 4) {
      // P = c0 I - w_1 D_1 - w_l D_l - w_{l+1} D_{l+1} with D_1 = T_0 / o read
      // from the T_0 buffer (coefficients known only after the first squaring)
      const float c0f = static_cast<float>(p.scal[pr.mat].c0);
      const float w1 = static_cast<float>(coef_at(p.coef, pr.mat, 1));
      const float inv = p.scal[pr.mat].inv_s2;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        float4 t = reinterpret_cast<const float4*>(P)[j];
        pv[4 * j] = t.x;
        pv[4 * j + 1] = t.y;
        pv[4 * j + 2] = t.z;
        pv[4 * j + 3] = t.w;
      }
#pragma unroll
      for (int j = 0; j < 32; ++j) pv[j] = fmaf(-w1, pv[j] * inv, (c0 + j == r) ? c0f : 0.f);
    } else if (p.p_mode >= 2) {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        float4 t = reinterpret_cast<const float4*>(P)[j];
        pv[4 * j] = t.x;
        pv[4 * j + 1] = t.y;
        pv[4 * j + 2] = t.z;
        pv[4 * j + 3] = t.w;
      }
    } else {
      const float c0f = p.p_mode == 1 ? static_cast<float>(p.scal[pr.mat].c0) : 0.f;
#pragma unroll
      for (int j = 0; j < 32; ++j) pv[j] = (c0 + j == r) ? c0f : 0.f;
    }
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const float dn = 2.0f * d[j] - v[j];  // D_{l+1} = 2 D_l - D_l^2
      v[j] = dn;
      pv[j] = fmaf(-w, dn, fmaf(-wp, d[j], pv[j]));
    }
    if (!p.final_pass) {
      if (p.p_mode != 0) {
#pragma unroll
        for (int j = 0; j < 8; ++j)
          reinterpret_cast<float4*>(P)[j] =
              make_float4(pv[4 * j], pv[4 * j + 1], pv[4 * j + 2], pv[4 * j + 3]);
      }
      if (p.write_lo) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const float hi = __half2float(__float2half_rn(v[j]));
          lo[j] = v[j] - hi;
          v[j] = hi;
        }
        store_sym<__half>(static_cast<__half*>(pr.out0), pr.ld_out, r, c0, v, mirror, st);
        store_sym<__half>(static_cast<__half*>(pr.out1), pr.ld_out, r, c0, lo, mirror, st);
      } else {
        store_sym<__half>(static_cast<__half*>(pr.out0), pr.ld_out, r, c0, v, mirror, st);
      }
    } else {
      if (p.p_split) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const float hi = __bfloat162float(__float2bfloat16_rn(pv[j]));
          lo[j] = pv[j] - hi;
          pv[j] = hi;
        }
        store_sym<__nv_bfloat16>(static_cast<__nv_bfloat16*>(pr.out0), pr.ld_out, r, c0, pv, mirror, st);
        store_sym<__nv_bfloat16>(static_cast<__nv_bfloat16*>(pr.out1), pr.ld_out, r, c0, lo, mirror, st);
      } else {
        store_sym<__nv_bfloat16>(static_cast<__nv_bfloat16*>(pr.out0), pr.ld_out, r, c0, pv, mirror, st);
      }
    }
  } else if constexpr (EPI == EPI_APPLY) {
    const float s = p.scal[pr.mat].inv_s;
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] *= s;
    store_out_bf16(pr, r, c0, v, st);
  } else if constexpr (EPI == EPI_NS_GRAM) {
    const float s2 = p.ns_step == 0 ? p.scal[pr.mat].inv_s2 : 1.0f;
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] *= s2;
    store_sym<__nv_bfloat16>(static_cast<__nv_bfloat16*>(pr.out0), pr.ld_out, r, c0, v, mirror, st);
  } else if constexpr (EPI == EPI_NS_SQR) {
    float s[32];
    load_b32(static_cast<const __nv_bfloat16*>(pr.aux0) + static_cast<int64_t>(r) * pr.ld_aux + c0, s);
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = fmaf(p.ns_c, v[j], p.ns_b * s[j]);
    store_sym<__nv_bfloat16>(static_cast<__nv_bfloat16*>(pr.out0), pr.ld_out, r, c0, v, mirror, st);
  } else if constexpr (EPI == EPI_NS_APPLY) {
    const float sc = p.ns_step == 0 ? p.scal[pr.mat].inv_s : 1.0f;
    float x[32];
    load_x_bf16(pr, r, c0, x, st);
    const float ka = p.ns_a * sc, kb = p.ns_bcoef * sc;
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = fmaf(ka, x[j], kb * v[j]);
    store_out_bf16(pr, r, c0, v, st);
  }
}

// ---------------------------------------------------------------- kernel

template <int NA, int NB, int EPI>
__global__ void __launch_bounds__(kThreads, 1) tc_gemm_kernel(const __grid_constant__ TcParams p) {
  using C = Cfg<NA, NB>;
  using PR = Products<NA, NB>;
  constexpr int S = C::stages;
  constexpr uint32_t kIsBf16 = (EPI == EPI_SQR) ? 0u : 1u;  // D_l are FP16, all else BF16
  constexpr uint16_t kPair = 0x3;                           // both CTAs of the cluster

  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* base_ptr = smem_raw + (base - raw);
  uint64_t* bars = reinterpret_cast<uint64_t*>(base_ptr + S * C::stage_bytes);
  const uint32_t bar0 = smem_u32(bars);
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (S + s); };
  auto tfull_bar = [&](int a) { return bar0 + 8u * (2 * S + a); };
  auto tempty_bar = [&](int a) { return bar0 + 8u * (2 * S + 2 + a); };
  const uint32_t drain_bar = bar0 + 8u * (2 * S + 4);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * S + 5);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  // A cluster of two CTAs computes the two 128-row halves of one 128 x 256
  // pair of tiles: both need the same B tile, which each CTA loads half of and
  // multicasts to both.
  const int crank = static_cast<int>(cluster_ctarank());
  const int cid = static_cast<int>(cluster_id_x());
  const int ncl = static_cast<int>(cluster_count_x());

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 2);  // freed by the MMAs of both CTAs (their B halves live here)
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(tfull_bar(a), 1);
      mbar_init(tempty_bar(a), 32 * kEpiWarps);
    }
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(smem_u32(tmem_slot), kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  cluster_sync();  // the peer's barriers are initialised before any multicast reaches them
  const uint32_t tmem_base = *tmem_slot;
  const unsigned long long tmo = p.wait_ms ? p.wait_ms * 1000000ull : kWaitTimeoutNs;

  if (warp == 0) {
    if (lane == 0) {
      // ------------------------------------------------ TMA producer
      int stage = 0;
      uint32_t phase = 0;
      uint32_t filled[6] = {0, 0, 0, 0, 0, 0};
      int cur_mat = 0;
      int last_prob = -1;
      bool ok = true;
      // testing aid: the first CTA loads nothing, so the waits of both CTAs of its cluster run out
      const int first = (p.inject && cid == 0 && crank == 0) ? p.n_items : cid;
      for (int it = first; it < p.n_items && ok; it += ncl) {
        const WorkItem wi = p.items[it];
        const TcProblem& pr = p.probs[wi.prob];
        cur_mat = pr.mat;
        if (wi.prob != last_prob) {
          last_prob = wi.prob;
#pragma unroll
          for (int a = 0; a < NA; ++a) tmap_acquire(&pr.mapA[a]);
#pragma unroll
          for (int b = 0; b < NB; ++b) tmap_acquire(&pr.mapB[b]);
        }
        const int a_mn = pr.a_mn, b_mn = pr.b_mn;
        const int n_kb = pr.n_kb;
        const int tm = wi.tm + crank;
        for (int kb = 0; kb < n_kb; ++kb) {
          if (!mbar_wait(empty_bar(stage), phase ^ 1u, abort_flag, tmo)) {
            ok = false;
            break;
          }
          const uint32_t fb = full_bar(stage);
          mbar_arrive_expect_tx(fb, C::stage_bytes);  // own A + both halves of B
          const uint32_t st = base + stage * C::stage_bytes;
          const int k0 = kb * BK;
#pragma unroll
          for (int a = 0; a < NA; ++a) {
            const uint32_t dst = st + a * kTileA;
            const void* m = &pr.mapA[a];
            if (!a_mn) {
              tma_load_2d(dst, m, fb, k0, tm * BM);
            } else {
              tma_load_2d(dst, m, fb, tm * BM, k0);
              tma_load_2d(dst + 8192, m, fb, tm * BM + 64, k0);
            }
          }
#pragma unroll
          for (int b = 0; b < NB; ++b) {
            const uint32_t dst = st + NA * kTileA + b * kTileB;
            const void* m = &pr.mapB[b];
            if (!b_mn) {
              // this CTA's half: rows [128 crank, 128 crank + 128) of the B tile
              tma_load_2d_mc(dst + 16384 * crank, m, fb, k0, wi.tn * BN + 128 * crank, kPair);
            } else {
              // this CTA's half: MN chunks 2 crank and 2 crank + 1 of the B tile
#pragma unroll
              for (int j = 2 * crank; j < 2 * crank + 2; ++j)
                tma_load_2d_mc(dst + 8192 * j, m, fb, wi.tn * BN + 64 * j, k0, kPair);
            }
          }
          ++filled[stage];
          if (++stage == S) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      if (!ok) {
        set_timeout(p.scal, cur_mat);
        // let the copies already issued land before the CTA exits
        for (int s = 0; s < S; ++s)
          if (filled[s]) mbar_wait_bounded(full_bar(s), (filled[s] - 1u) & 1u, tmo);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ------------------------------------------------ MMA issuer
      int stage = 0;
      uint32_t phase = 0;
      int local = 0;
      int cur_mat = 0;
      bool ok = true;
      for (int it = cid; it < p.n_items && ok; it += ncl, ++local) {
        const WorkItem wi = p.items[it];
        const TcProblem& pr = p.probs[wi.prob];
        cur_mat = pr.mat;
        const int acc = local & 1;
        const uint32_t acc_phase = (static_cast<uint32_t>(local) >> 1) & 1u;
        if (!mbar_wait(tempty_bar(acc), acc_phase ^ 1u, abort_flag, tmo)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + static_cast<uint32_t>(acc * BN);
        const uint32_t a_mn = static_cast<uint32_t>(pr.a_mn), b_mn = static_cast<uint32_t>(pr.b_mn);
        const uint32_t idesc = idesc_f16(kIsBf16, BM, BN, a_mn, b_mn);
        const int n_kb = pr.n_kb;
        for (int kb = 0; kb < n_kb; ++kb) {
          if (!mbar_wait(full_bar(stage), phase, abort_flag, tmo)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t st = base + stage * C::stage_bytes;
#pragma unroll
          for (int k = 0; k < BK / 16; ++k) {
#pragma unroll
            for (int q = 0; q < PR::n; ++q) {
              const uint32_t sa = st + PR::a(q) * kTileA;
              const uint32_t sb = st + NA * kTileA + PR::b(q) * kTileB;
              const uint64_t ad = a_mn ? sdesc_sw128(sa + k * 2048, 8192, 1024)
                                       : sdesc_sw128(sa + k * 32, 16, 1024);
              const uint64_t bd = b_mn ? sdesc_sw128(sb + k * 2048, 8192, 1024)
                                       : sdesc_sw128(sb + k * 32, 16, 1024);
              umma_f16(d_tmem, ad, bd, idesc, (kb | k | q) != 0 ? 1u : 0u);
            }
          }
          // frees the stage in both CTAs once these MMAs have read it
          umma_commit_mc(empty_bar(stage), kPair);
          if (++stage == S) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (!ok) break;
        umma_commit(tfull_bar(acc));  // accumulator ready for the epilogue
      }
      if (!ok) set_timeout(p.scal, cur_mat);
      // make sure no MMA is still writing TMEM or reading shared memory
      umma_commit(drain_bar);
      mbar_wait_bounded(drain_bar, 0, tmo);
    }
  } else {
    // -------------------------------------------------- epilogue (warps 2..9)
    float* stage = reinterpret_cast<float*>(base_ptr + S * C::stage_bytes + 256) + (warp - 2) * 32 * kStageLd;
    const int q = warp & 3;            // TMEM lane quadrant this warp may access
    const int half = (warp - 2) >> 2;  // which 128 of the tile's 256 columns
    const int row_in_tile = q * 32 + lane;
    int local = 0;
    for (int it = cid; it < p.n_items; it += ncl, ++local) {
      const WorkItem wi = p.items[it];
      const TcProblem& pr = p.probs[wi.prob];
      const int acc = local & 1;
      const uint32_t acc_phase = (static_cast<uint32_t>(local) >> 1) & 1u;
      // one lane waits, the warp follows its verdict (tcgen05.ld needs a converged warp)
      int ready = 0;
      if (lane == 0) ready = mbar_wait(tfull_bar(acc), acc_phase, abort_flag, tmo) ? 1 : 0;
      ready = __shfl_sync(0xffffffffu, ready, 0);
      if (!ready) {
        if (lane == 0) set_timeout(p.scal, pr.mat);
        break;
      }
      tc_fence_after();
      const uint32_t tbase = tmem_base + (static_cast<uint32_t>(q * 32) << 16) + static_cast<uint32_t>(acc * BN);
      const int r = (wi.tm + crank) * BM + row_in_tile;
      EpiAcc ea{0.f, 0.f};
#pragma unroll 1
      for (int ch = half * (BN / 64); ch < (half + 1) * (BN / 64); ++ch) {
        uint32_t u[32];
        IFNSO_TMEM_LD32(tbase + static_cast<uint32_t>(ch * 32), u);
        IFNSO_TMEM_WAIT_LD(u);
        float v[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = u2f(u[j]);
        epilogue_chunk<EPI>(p, pr, wi, r, wi.tn * BN + ch * 32, v, ea, stage);
      }
      tc_fence_before();
      mbar_arrive(tempty_bar(acc));
      if constexpr (EPI == EPI_GRAM) {
        float ss = ea.ss, tr = ea.tr;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          ss += __shfl_xor_sync(0xffffffffu, ss, o);
          tr += __shfl_xor_sync(0xffffffffu, tr, o);
        }
        if (lane == 0) {
          const double wgt = (wi.flags & 1) ? 1.0 : 2.0;  // off-diagonal blocks stand for two
          atomicAdd(&p.scal[pr.mat].o2, wgt * static_cast<double>(ss));
          if (tr != 0.f) atomicAdd(&p.scal[pr.mat].trace, static_cast<double>(tr));
        }
      }
      if constexpr (EPI == EPI_SQR) {
        if (p.feat) {
          const float ss = warp_reduce_sum(ea.ss);
          if (lane == 0)
            atomicAdd(&p.scal[pr.mat].spare[0], ((wi.flags & 1) ? 1.0 : 2.0) * static_cast<double>(ss));
        }
      }
    }
  }

  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, kTmemCols);
  }
  // neither CTA leaves while the other may still multicast into it or arrive on its barriers
  cluster_sync();
}

template <int NA, int NB, int EPI>
cudaError_t launch_one(const TcParams& p, int max_clusters, cudaStream_t s) {
  using C = Cfg<NA, NB>;
  auto kern = tc_gemm_kernel<NA, NB, EPI>;
  static int active_clusters = 0;  // per process and instantiation
  if (active_clusters == 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t q = {};
    cudaLaunchAttribute qa[1];
    qa[0].id = cudaLaunchAttributeClusterDimension;
    qa[0].val.clusterDim.x = 2;
    qa[0].val.clusterDim.y = 1;
    qa[0].val.clusterDim.z = 1;
    q.gridDim = dim3(2, 1, 1);
    q.blockDim = dim3(kThreads, 1, 1);
    q.dynamicSmemBytes = C::smem;
    q.attrs = qa;
    q.numAttrs = 1;
    int n = 0;
    e = cudaOccupancyMaxActiveClusters(&n, kern, &q);
    if (e != cudaSuccess) return e;
    active_clusters = n > 0 ? n : 1;
  }
  int clusters = active_clusters < max_clusters ? active_clusters : max_clusters;
  if (clusters > p.n_items) clusters = p.n_items;
  if (clusters < 1) clusters = 1;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(2 * clusters, 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = C::smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, kern, p);
  count_launch();
  return e;
}

}  // namespace

int tc_smem_bytes(int na, int nb) {
  if (na == 1 && nb == 1) return Cfg<1, 1>::smem;
  if (na == 2 && nb == 2) return Cfg<2, 2>::smem;
  if (na == 2 && nb == 1) return Cfg<2, 1>::smem;
  return -1;
}

cudaError_t tc_launch(int epi, int na, int nb, const TcParams& p, int max_clusters, cudaStream_t s) {
  if (p.n_items == 0) return cudaSuccess;
  switch (epi) {
    case EPI_GRAM:
      return launch_one<1, 1, EPI_GRAM>(p, max_clusters, s);
    case EPI_SQR:
      if (na == 2) return launch_one<2, 2, EPI_SQR>(p, max_clusters, s);
      return launch_one<1, 1, EPI_SQR>(p, max_clusters, s);
    case EPI_APPLY:
      if (na == 2) return launch_one<2, 1, EPI_APPLY>(p, max_clusters, s);
      return launch_one<1, 1, EPI_APPLY>(p, max_clusters, s);
    case EPI_NS_GRAM:
      return launch_one<1, 1, EPI_NS_GRAM>(p, max_clusters, s);
    case EPI_NS_SQR:
      return launch_one<1, 1, EPI_NS_SQR>(p, max_clusters, s);
    case EPI_NS_APPLY:
      return launch_one<1, 1, EPI_NS_APPLY>(p, max_clusters, s);
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace ifnso
