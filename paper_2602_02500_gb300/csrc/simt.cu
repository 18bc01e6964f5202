// SIMT kernels of the IFNSO library: the split-K Frobenius norm, the
// per-matrix scalars (o, 1/sqrt(o), the D-basis identity weight in FP64),
// the elementwise initialisation D_1 = T_0/o, P = (1 + sum w) I - w_1 D_1,
// the FP32 GEMM that carries every product of FP32 plans, and the momentum
// step of a Muon update around the orthogonalization.
#include <algorithm>

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "common.cuh"

namespace ifnso {

namespace {

constexpr int kDevZero = 1;       // IFNSO_DEV_ZERO_INPUT
constexpr int kDevNonFinite = 2;  // IFNSO_DEV_NONFINITE

__device__ __forceinline__ float block_sum(float v, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  float s = 0.f;
  if (warp == 0) {
    s = lane < static_cast<int>(blockDim.x >> 5) ? red[lane] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  return s;  // valid in thread 0
}

// ---------------------------------------------------------------- norm
// ||M||_F^2 of every matrix: block (x, m) sums the squares of rows
// [x * chunk, (x + 1) * chunk) of matrix m in FP32 and adds its partial to
// out[m * out_stride] in FP64.  Rows whose start is 16-byte aligned are read
// as 16-byte vectors.
__global__ void __launch_bounds__(256) k_norm2(const MatInfo* mats, int bf16, double* out,
                                               int64_t out_stride) {
  __shared__ float red[32];
  const MatInfo& mi = mats[blockIdx.y];
  const int64_t rows = mi.rows, cols = mi.cols, ld = mi.ld;
  const int64_t chunk = (rows + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = blockIdx.x * chunk;
  const int64_t r1 = r0 + chunk < rows ? r0 + chunk : rows;
  float acc = 0.f;
  if (bf16) {
    const __nv_bfloat16* A = static_cast<const __nv_bfloat16*>(mi.in);
    const bool vec = (ld % 8 == 0) && (cols % 8 == 0) && ((reinterpret_cast<uintptr_t>(A) & 15) == 0);
    if (vec) {
      const int64_t c8 = cols / 8;
      const int64_t n = (r1 - r0) * c8;
      for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
        const int64_t r = r0 + e / c8, c = (e % c8) * 8;
        const uint4 u = *reinterpret_cast<const uint4*>(A + r * ld + c);
        const __nv_bfloat162* h2 = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const float2 f = __bfloat1622float2(h2[t]);
          acc = fmaf(f.x, f.x, acc);
          acc = fmaf(f.y, f.y, acc);
        }
      }
    } else {
      const int64_t n = (r1 - r0) * cols;
      for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
        const float f = __bfloat162float(A[(r0 + e / cols) * ld + e % cols]);
        acc = fmaf(f, f, acc);
      }
    }
  } else {
    const float* A = static_cast<const float*>(mi.in);
    const int64_t n = (r1 - r0) * cols;
    for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
      const float f = A[(r0 + e / cols) * ld + e % cols];
      acc = fmaf(f, f, acc);
    }
  }
  const float s = block_sum(acc, red);
  if (threadIdx.x == 0 && r0 < rows) atomicAdd(out + blockIdx.y * out_stride, static_cast<double>(s));
}

// ---------------------------------------------------------------- E4M3 Gram input
// max |M_ij| of every matrix (block (x, m): rows [x chunk, (x + 1) chunk) of
// matrix m; BF16), as the bit pattern of a non-negative float, into
// MatScalars::amax of matrix m.  Rows whose start is 16-byte aligned are read
// as 16-byte vectors.
__global__ void __launch_bounds__(256) k_amax(const MatInfo* mats, MatScalars* scal) {
  __shared__ float red[32];
  const MatInfo& mi = mats[blockIdx.y];
  const int64_t rows = mi.rows, cols = mi.cols, ld = mi.ld;
  const int64_t chunk = (rows + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = blockIdx.x * chunk;
  const int64_t r1 = r0 + chunk < rows ? r0 + chunk : rows;
  const __nv_bfloat16* A = static_cast<const __nv_bfloat16*>(mi.in);
  const bool vec = (ld % 8 == 0) && ((reinterpret_cast<uintptr_t>(A) & 15) == 0);
  const int64_t c8 = vec ? cols / 8 * 8 : 0;  // columns read as vectors
  float mx = 0.f;
  for (int64_t r = r0; r < r1; ++r) {
    const __nv_bfloat16* row = A + r * ld;
    for (int64_t c = threadIdx.x * 8; c < c8; c += blockDim.x * 8) {
      const uint4 u = *reinterpret_cast<const uint4*>(row + c);
      const __nv_bfloat162* h2 = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const float2 f = __bfloat1622float2(h2[t]);
        mx = fmaxf(mx, fmaxf(fabsf(f.x), fabsf(f.y)));
      }
    }
    for (int64_t c = c8 + threadIdx.x; c < cols; c += blockDim.x) mx = fmaxf(mx, fabsf(__bfloat162float(row[c])));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[warp] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    float m = 0.f;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
    atomicMax(&scal[blockIdx.y].amax, __float_as_uint(m));
  }
}

// Four values of A s in E4M3 (round to nearest even, saturating at +-448),
// packed little-endian into 32 bits.
__device__ __forceinline__ uint32_t e4m3x4(float a, float b, float c, float d) {
  const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE, __NV_E4M3);
  const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(c, d), __NV_SATFINITE, __NV_E4M3);
  return (lo & 0xFFFFu) | (hi << 16);
}

// A s in E4M3, K-major: A = M for a wide matrix, M^T for a tall one.  Block
// (x, y, m) writes output rows [32 y, 32 y + 32) and columns
// [128 x, 128 x + 128) of matrix m: a wide matrix is converted row by row
// (each thread 4 consecutive values, one 32-bit store); a tall one goes
// through a 128 x 33 tile so that both its reads and its writes are along
// rows of their matrices.
// The FP16 copy M s of matrix blockIdx.y in M's own layout (an elementwise
// cast: the product reads it through the same view as the BF16 input), 8
// values per thread and step; rows of M are 16-byte aligned (the input's TMA
// views require it).  BF16 values scaled by a power of two convert exactly
// while they stay within the FP16 normal range.
__global__ void __launch_bounds__(256) k_cast_f16(const MatInfo* mats, const MatScalars* scal) {
  const MatInfo& mi = mats[blockIdx.y];
  if (mi.on_chip || !mi.a16) return;
  const float s = f16_copy_scale(scal[blockIdx.y].trace);
  const int64_t vpr = (mi.cols + 7) / 8;  // 8-value pieces per row
  const int64_t n = mi.rows * vpr;
  const __nv_bfloat16* M = static_cast<const __nv_bfloat16*>(mi.in);
  __half* D = static_cast<__half*>(mi.a16);
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = i / vpr, c = (i - r * vpr) * 8;
    const __nv_bfloat16* src = M + r * mi.ld + c;
    __half* dst = D + r * mi.a16ld + c;
    if (c + 8 <= mi.cols) {
      const uint4 u = *reinterpret_cast<const uint4*>(src);
      const __nv_bfloat162* e = reinterpret_cast<const __nv_bfloat162*>(&u);
      uint4 o;
      __half2* h = reinterpret_cast<__half2*>(&o);
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const float2 f = __bfloat1622float2(e[t]);
        h[t] = __floats2half2_rn(f.x * s, f.y * s);
      }
      *reinterpret_cast<uint4*>(dst) = o;
    } else {
      for (int64_t t = 0; c + t < mi.cols; ++t) dst[t] = __float2half_rn(__bfloat162float(src[t]) * s);
    }
  }
}

__global__ void __launch_bounds__(256) k_cast_e4m3(const MatInfo* mats, const MatScalars* scal) {
  __shared__ float tile[128][33];
  const MatInfo& mi = mats[blockIdx.z];
  const int h = mi.h, w = mi.w;
  const int i0 = blockIdx.y * 32, k0 = blockIdx.x * 128;
  if (i0 >= h || k0 >= w) return;
  const __nv_bfloat16* M = static_cast<const __nv_bfloat16*>(mi.in);
  const float s = e4m3_scale(scal[blockIdx.z].amax);
  const int t = threadIdx.x;
  // output row i0 + (t >> 3) (+ 32 / 8 per step), columns k0 + 4 (t & 7) + 32 j
  if (!mi.trans) {
    for (int rr = t >> 5; rr < 32; rr += 8) {
      const int oi = i0 + rr;
      if (oi >= h) break;
      const int ok = k0 + 4 * (t & 31);
      if (ok >= w) continue;
      const __nv_bfloat16* src = M + static_cast<int64_t>(oi) * mi.ld + ok;
      float v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) v[q] = (ok + q < w) ? __bfloat162float(src[q]) * s : 0.f;
      uint8_t* dst = mi.a8 + static_cast<int64_t>(oi) * mi.a8ld + ok;
      const uint32_t packed = e4m3x4(v[0], v[1], v[2], v[3]);
      if (ok + 4 <= w) {
        *reinterpret_cast<uint32_t*>(dst) = packed;  // a8ld and ok are multiples of 4
      } else {
        for (int q = 0; ok + q < w; ++q) dst[q] = static_cast<uint8_t>(packed >> (8 * q));
      }
    }
    return;
  }
  // tall: source rows k0..k0+127 of M, columns i0..i0+31
  for (int r = t >> 5; r < 128; r += 8) {
    const int64_t sr = k0 + r, sc = i0 + (t & 31);
    tile[r][t & 31] = (sr < mi.rows && sc < mi.cols) ? __bfloat162float(M[sr * mi.ld + sc]) : 0.f;
  }
  __syncthreads();
  for (int rr = t >> 5; rr < 32; rr += 8) {
    const int oi = i0 + rr;
    const int kk = 4 * (t & 31);
    const int ok = k0 + kk;
    if (oi >= h || ok >= w) continue;
    const uint32_t packed = e4m3x4(tile[kk][rr] * s, tile[kk + 1][rr] * s, tile[kk + 2][rr] * s,
                                   tile[kk + 3][rr] * s);
    uint8_t* dst = mi.a8 + static_cast<int64_t>(oi) * mi.a8ld + ok;
    if (ok + 4 <= w) {
      *reinterpret_cast<uint32_t*>(dst) = packed;
    } else {
      for (int q = 0; ok + q < w; ++q) dst[q] = static_cast<uint8_t>(packed >> (8 * q));
    }
  }
}

// ---------------------------------------------------------------- scalars
// One thread per matrix: the squared scale s2 (o = sqrt(sum T_0^2) for the
// Gram scaling of Sec. 2, ||A||_F^2 = tr T_0 for the Frobenius scaling), its
// FP32 reciprocals, the D-basis identity weight c0 = 1 + sum_{l=1}^L w_l in
// FP64, and the zero / non-finite status bits.
__global__ void k_scalars(const MatInfo* mats, int count, MatScalars* scal, CoefTable coef, int L, int frob) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= count) return;
  if (mats && mats[m].on_chip) return;  // the on-chip path wrote this matrix's scalars
  MatScalars& s = scal[m];
  const double s2 = frob ? s.trace : sqrt(s.o2);
  int st = s.status;
  double c0 = 1.0;
  for (int l = 1; l <= L; ++l) c0 += coef_at(coef, m, l);
  const bool fin = isfinite(s2) && isfinite(c0);
  if (!fin) st |= kDevNonFinite;
  if (fin && s2 == 0.0) st |= kDevZero;
  const bool pos = fin && s2 > 0.0;
  s.s2 = s2;
  s.c0 = c0;
  s.inv_s2 = pos ? static_cast<float>(1.0 / s2) : 0.f;
  s.inv_s = pos ? static_cast<float>(1.0 / sqrt(s2)) : 0.f;
  s.status = st;
}

// Gelfand's bound with q = 2 (Eq. gelfand_formula): the scalars of Gram
// scaling hold o = ||T_0||_F, and the norm pass summed ||(T_0/o)^2||_F^2 into
// spare[0]; o <- ||T_0^2||_F^(1/2) = o spare[0]^(1/4), in FP64.  Zero,
// non-finite and flagged matrices keep their scalars.
__global__ void k_gelfand(int count, MatScalars* scal) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= count) return;
  MatScalars& s = scal[m];
  const double q = s.spare[0];
  s.spare[0] = 0.0;
  if (s.status != 0 || !(s.s2 > 0.0) || !(q > 0.0) || !isfinite(q)) return;
  const double s2 = s.s2 * sqrt(sqrt(q));
  s.s2 = s2;
  s.inv_s2 = static_cast<float>(1.0 / s2);
  s.inv_s = static_cast<float>(1.0 / sqrt(s2));
}

// ---------------------------------------------------------------- prep
// Elementwise over the h_pad x h_pad buffers of every matrix:
//   d = T_0 * (1/s2)                       (D_1 = T_0 / o, the scaled Gram)
//   P = c0 [i == j] - w_1 d                (Y' accumulated in the D basis)
// BF16 plans store D_1 as FP16 (hi, and lo = d - hi when split) in D buffer
// 0; their first squaring writes P (FP32, in place of T_0).  For L = 1 there
// is no squaring: P itself is written as BF16 (hi, lo) into D buffer 0.
// FP32 plans store D_1 in FP32 in D buffer 0 and P in place of T_0.
__global__ void __launch_bounds__(256) k_prep(const MatInfo* mats, MatScalars* scal, CoefTable coef,
                                              int L, int split, int f32, int d_only, int write_p) {
  const int m = blockIdx.y;
  const MatInfo& mi = mats[m];
  if (mi.on_chip) return;  // computed by the on-chip path
  const int64_t hp = mi.hpad;
  const int64_t n = hp * hp;
  const float inv = scal[m].inv_s2;
  const float c0 = static_cast<float>(scal[m].c0);
  const float w1 = static_cast<float>(coef_at(coef, m, 1));
  float* gp = mi.gp;
  // 8 consecutive elements of one row per step (h_pad is a multiple of 256):
  // two 16-byte loads of T_0, 16-byte stores of every output.  FP32 plans
  // cover the whole h_pad x h_pad buffer with a grid-stride loop; the
  // tensor-core path stores symmetric intermediates on the 256 x 256 blocks on
  // and above the diagonal only, and there each CTA takes one such block.
  const int64_t row8 = hp / 8;
  const int nb = static_cast<int>(hp / 256);
  int bi = 0, bj = 0;
  if (!f32) {
    int t = blockIdx.x;
    if (t >= nb * (nb + 1) / 2) return;
    while (t >= nb - bi) {  // block row bi holds blocks bi..nb-1
      t -= nb - bi;
      ++bi;
    }
    bj = bi + t;
  }
  const int64_t steps = f32 ? n / 8 : 256 * 32;
  const int64_t first = f32 ? blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x : threadIdx.x;
  const int64_t stride = f32 ? static_cast<int64_t>(gridDim.x) * blockDim.x : blockDim.x;
  for (int64_t e8 = first; e8 < steps; e8 += stride) {
    int64_t i, j0;
    if (f32) {
      i = e8 / row8;
      j0 = (e8 - i * row8) * 8;
    } else {
      i = 256 * static_cast<int64_t>(bi) + (e8 >> 5);
      j0 = 256 * static_cast<int64_t>(bj) + (e8 & 31) * 8;
    }
    const int64_t e = i * hp + j0;
    const float4 g0 = reinterpret_cast<const float4*>(gp + e)[0];
    const float4 g1 = reinterpret_cast<const float4*>(gp + e)[1];
    const float g[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
    float d[8], p[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      d[t] = g[t] * inv;
      p[t] = fmaf(-w1, d[t], (j0 + t == i) ? c0 : 0.f);
    }
    if (f32) {
      float4* dd = reinterpret_cast<float4*>(static_cast<float*>(mi.d[0]) + e);
      dd[0] = make_float4(d[0], d[1], d[2], d[3]);
      dd[1] = make_float4(d[4], d[5], d[6], d[7]);
      if (!d_only) {
        reinterpret_cast<float4*>(gp + e)[0] = make_float4(p[0], p[1], p[2], p[3]);
        reinterpret_cast<float4*>(gp + e)[1] = make_float4(p[4], p[5], p[6], p[7]);
      }
    } else if (L == 1 && !d_only) {
      uint4 uh, ul;
      __nv_bfloat162* h2 = reinterpret_cast<__nv_bfloat162*>(&uh);
      __nv_bfloat162* l2 = reinterpret_cast<__nv_bfloat162*>(&ul);
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        h2[t] = __floats2bfloat162_rn(p[2 * t], p[2 * t + 1]);
        const float2 hf = __bfloat1622float2(h2[t]);
        l2[t] = __floats2bfloat162_rn(p[2 * t] - hf.x, p[2 * t + 1] - hf.y);
      }
      *reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(mi.d[0]) + e) = uh;
      if (split) *reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(mi.d[1]) + e) = ul;
    } else {
      uint4 uh, ul;
      __half2* h2 = reinterpret_cast<__half2*>(&uh);
      __half2* l2 = reinterpret_cast<__half2*>(&ul);
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        h2[t] = __floats2half2_rn(d[2 * t], d[2 * t + 1]);
        const float2 hf = __half22float2(h2[t]);
        l2[t] = __floats2half2_rn(d[2 * t] - hf.x, d[2 * t + 1] - hf.y);
      }
      *reinterpret_cast<uint4*>(static_cast<__half*>(mi.d[0]) + e) = uh;
      if (split) *reinterpret_cast<uint4*>(static_cast<__half*>(mi.d[1]) + e) = ul;
      if (write_p) {
        // P = c0 I - w_1 D_1 in FP32, over T_0 (the squarings add their terms to it)
        reinterpret_cast<float4*>(gp + e)[0] = make_float4(p[0], p[1], p[2], p[3]);
        reinterpret_cast<float4*>(gp + e)[1] = make_float4(p[4], p[5], p[6], p[7]);
      }
      // (otherwise the first squaring writes P, with its first two terms)
    }
  }
}

// ---------------------------------------------------------------- FP32 GEMM
// C(i, j) = sum_k A(i, k) B(j, k) over 64 x 64 tiles, 16-wide K slices,
// 256 threads with 4 x 4 outputs each, followed by the epilogue of the pass.
template <int EPI>
__global__ void __launch_bounds__(256) k_sgemm(const SgParams p) {
  const SgProblem& pr = p.probs[blockIdx.z];
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  if (m0 >= pr.M || n0 >= pr.N) return;
  __shared__ float As[16][68];
  __shared__ float Bs[16][68];
  __shared__ float red[32];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
  const bool a_kc = pr.sa1 == 1;  // A contiguous along k
  const bool b_kc = pr.sb1 == 1;
  for (int k0 = 0; k0 < pr.K; k0 += 16) {
    for (int e = threadIdx.x; e < 1024; e += 256) {
      int i, k;
      if (a_kc) { i = e >> 4; k = e & 15; } else { i = e & 63; k = e >> 6; }
      const int gi = m0 + i, gk = k0 + k;
      As[k][i] = (gi < pr.a_rows && gk < pr.K) ? pr.A[gi * pr.sa0 + gk * pr.sa1] : 0.f;
      int j, kk;
      if (b_kc) { j = e >> 4; kk = e & 15; } else { j = e & 63; kk = e >> 6; }
      const int gj = n0 + j, gkk = k0 + kk;
      Bs[kk][j] = (gj < pr.b_rows && gkk < pr.K) ? pr.B[gj * pr.sb0 + gkk * pr.sb1] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      float av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[k][ty * 4 + a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bs[k][tx * 4 + b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
  float ss = 0.f, tr = 0.f;
  double nn = 0.0;
  const int m = pr.mat;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int i = m0 + ty * 4 + a, j = n0 + tx * 4 + b;
      if (i >= pr.M || j >= pr.N) continue;
      float v = acc[a][b];
      if constexpr (EPI == EPI_GRAM) {
        pr.pacc[i * pr.ld_aux + j] = v;
        ss = fmaf(v, v, ss);
        if (i == j) tr += v;
      } else if constexpr (EPI == EPI_SQR_NORM) {
        // (D_1^2)_ij with D_1 = T_0 / o; the squares are summed in FP64 below
        nn = fma(static_cast<double>(v), static_cast<double>(v), nn);
      } else if constexpr (EPI == EPI_SQR) {
        const int64_t o = i * pr.ld_aux + j;
        const float dn = 2.0f * pr.aux0[o] - v;
        const float w = static_cast<float>(coef_at(p.coef, m, p.coef_l));
        pr.pacc[o] = fmaf(-w, dn, pr.pacc[o]);
        if (!p.final_pass) pr.out0[i * pr.ld_out + j] = dn;
      } else if constexpr (EPI == EPI_APPLY || EPI == EPI_NS_APPLY) {
        const int oi = pr.out_trans ? j : i, oj = pr.out_trans ? i : j;
        if (oi >= pr.rows_out || oj >= pr.cols_out) continue;
        float r;
        if constexpr (EPI == EPI_APPLY) {
          r = v * p.scal[m].inv_s;
        } else {
          const float sc = p.ns_step == 0 ? p.scal[m].inv_s : 1.0f;
          const float x = pr.aux0[oi * pr.ld_aux + oj];
          r = fmaf(p.ns_a * sc, x, p.ns_bcoef * sc * v);
        }
        pr.out0[oi * pr.ld_out + oj] = r;
      } else if constexpr (EPI == EPI_NS_GRAM) {
        const float s2 = p.ns_step == 0 ? p.scal[m].inv_s2 : 1.0f;
        pr.out0[i * pr.ld_out + j] = v * s2;
      } else if constexpr (EPI == EPI_NS_SQR) {
        const float sv = pr.aux0[i * pr.ld_aux + j];
        pr.out0[i * pr.ld_out + j] = fmaf(p.ns_c, v, p.ns_b * sv);
      }
    }
  }
  if constexpr (EPI == EPI_SQR_NORM) {
    // per-block FP64 sum of the squares (FP32 partials would lose digits here)
    for (int o = 16; o > 0; o >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&p.scal[m].spare[0], nn);
  }
  if constexpr (EPI == EPI_GRAM) {
    const float s = block_sum(ss, red);
    const float t = block_sum(tr, red);
    if (threadIdx.x == 0) {
      atomicAdd(&p.scal[m].o2, static_cast<double>(s));
      if (t != 0.f) atomicAdd(&p.scal[m].trace, static_cast<double>(t));
    }
  }
}

// Muon's momentum step for one matrix, 8 consecutive elements of a row per
// thread (cols and ldg multiples of 8 are not required: the row tail goes
// element by element).  M <- beta M + G; U <- G + beta M (nesterov) or M.
__global__ void __launch_bounds__(256) k_muon_momentum(const __nv_bfloat16* __restrict__ g, int64_t ldg,
                                                      float* __restrict__ m, __nv_bfloat16* __restrict__ u,
                                                      int64_t rows, int64_t cols, float beta, int nesterov) {
  const int64_t row8 = (cols + 7) / 8;
  for (int64_t e8 = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e8 < rows * row8;
       e8 += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = e8 / row8, j0 = (e8 - i * row8) * 8;
    const __nv_bfloat16* gr = g + i * ldg + j0;
    float* mr = m + i * cols + j0;
    __nv_bfloat16* ur = u + i * ldg + j0;
    if (j0 + 8 <= cols && (ldg & 7) == 0 && (cols & 3) == 0) {
      const uint4 gv = *reinterpret_cast<const uint4*>(gr);
      const __nv_bfloat162* g2 = reinterpret_cast<const __nv_bfloat162*>(&gv);
      float4 m0 = reinterpret_cast<const float4*>(mr)[0], m1 = reinterpret_cast<const float4*>(mr)[1];
      float mv[8] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w};
      uint4 uv;
      __nv_bfloat162* u2 = reinterpret_cast<__nv_bfloat162*>(&uv);
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const float2 gf = __bfloat1622float2(g2[t]);
        mv[2 * t] = fmaf(beta, mv[2 * t], gf.x);
        mv[2 * t + 1] = fmaf(beta, mv[2 * t + 1], gf.y);
        const float a = nesterov ? fmaf(beta, mv[2 * t], gf.x) : mv[2 * t];
        const float b = nesterov ? fmaf(beta, mv[2 * t + 1], gf.y) : mv[2 * t + 1];
        u2[t] = __floats2bfloat162_rn(a, b);
      }
      reinterpret_cast<float4*>(mr)[0] = make_float4(mv[0], mv[1], mv[2], mv[3]);
      reinterpret_cast<float4*>(mr)[1] = make_float4(mv[4], mv[5], mv[6], mv[7]);
      *reinterpret_cast<uint4*>(ur) = uv;
    } else {
      for (int64_t j = 0; j < 8 && j0 + j < cols; ++j) {
        const float gf = __bfloat162float(gr[j]);
        const float mv = fmaf(beta, mr[j], gf);
        mr[j] = mv;
        ur[j] = __float2bfloat16_rn(nesterov ? fmaf(beta, mv, gf) : mv);
      }
    }
  }
}

}  // namespace

cudaError_t launch_muon_momentum(const void* g, int64_t ldg, float* m, void* u, int64_t rows, int64_t cols,
                                 float beta, int nesterov, cudaStream_t s) {
  const int64_t n8 = rows * ((cols + 7) / 8);
  const int grid = static_cast<int>(std::min<int64_t>((n8 + 255) / 256, 4096));
  k_muon_momentum<<<grid, 256, 0, s>>>(static_cast<const __nv_bfloat16*>(g), ldg, m, static_cast<__nv_bfloat16*>(u),
                                       rows, cols, beta, nesterov);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_norm2(const MatInfo* d_mats, int count, int bf16, double* out,
                         int64_t out_stride, int grid_x, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  dim3 grid(grid_x, count);
  k_norm2<<<grid, 256, 0, s>>>(d_mats, bf16, out, out_stride);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_scalars(const MatInfo* d_mats, int count, MatScalars* scal, CoefTable coef, int L,
                           int scale_frob, int, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  k_scalars<<<(count + 127) / 128, 128, 0, s>>>(d_mats, count, scal, coef, L, scale_frob);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_prep(const MatInfo* d_mats, int count, int hpad_max, MatScalars* scal,
                        CoefTable coef, int L, int split, int f32, cudaStream_t s, int d_only, int write_p) {
  if (count == 0) return cudaSuccess;
  const int64_t n = static_cast<int64_t>(hpad_max) * hpad_max;
  int gx = static_cast<int>((n + 256 * 8 - 1) / (256 * 8));
  if (gx > 4096) gx = 4096;
  if (!f32) {
    const int nb = hpad_max / 256;  // one CTA per upper 256 x 256 block
    gx = nb * (nb + 1) / 2;
  }
  dim3 grid(gx, count);
  k_prep<<<grid, 256, 0, s>>>(d_mats, scal, coef, L, split, f32, d_only, write_p);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_gelfand(int count, MatScalars* scal, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  k_gelfand<<<(count + 127) / 128, 128, 0, s>>>(count, scal);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_amax(const MatInfo* d_mats, int count, MatScalars* scal, int grid_x, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  k_amax<<<dim3(grid_x, count), 256, 0, s>>>(d_mats, scal);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_cast_e4m3(const MatInfo* d_mats, int count, int max_h, int max_w, MatScalars* scal,
                             cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  k_cast_e4m3<<<dim3((max_w + 127) / 128, (max_h + 31) / 32, count), 256, 0, s>>>(d_mats, scal);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_cast_f16(const MatInfo* d_mats, int count, const MatScalars* scal, int grid_x, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_cast_f16<<<dim3(grid_x, count), 256, 0, s>>>(d_mats, scal);
  count_launch();
  return cudaGetLastError();
}

cudaError_t sg_launch(int epi, const SgParams& p, int count, int max_m, int max_n, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  dim3 grid((max_n + 63) / 64, (max_m + 63) / 64, count);
  switch (epi) {
    case EPI_GRAM: k_sgemm<EPI_GRAM><<<grid, 256, 0, s>>>(p); break;
    case EPI_SQR: k_sgemm<EPI_SQR><<<grid, 256, 0, s>>>(p); break;
    case EPI_APPLY: k_sgemm<EPI_APPLY><<<grid, 256, 0, s>>>(p); break;
    case EPI_SQR_NORM: k_sgemm<EPI_SQR_NORM><<<grid, 256, 0, s>>>(p); break;
    case EPI_NS_GRAM: k_sgemm<EPI_NS_GRAM><<<grid, 256, 0, s>>>(p); break;
    case EPI_NS_SQR: k_sgemm<EPI_NS_SQR><<<grid, 256, 0, s>>>(p); break;
    case EPI_NS_APPLY: k_sgemm<EPI_NS_APPLY><<<grid, 256, 0, s>>>(p); break;
    default: return cudaErrorInvalidValue;
  }
  count_launch();
  return cudaGetLastError();
}

}  // namespace ifnso

// ====================================================================
// Frobenius norm without any device allocation.
//
// ifnso_frobenius_norm2 keeps its per-matrix descriptors in device memory it
// allocates with cudaMalloc on first use.  Some callers cannot allow that:
// hosts that own all device memory through their own pool (a framework's
// caching allocator, an inference server's arena) and do not want a library
// to take memory behind their back or fail with out-of-memory mid-step, and
// latency-critical code for which the device-wide synchronisation of
// cudaMalloc / cudaFree is not acceptable.  This variant runs the same
// k_norm2 kernel with its descriptors in a fixed array that lives in the
// library image itself.
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "ifnso.h"

namespace ifnso {
namespace {

constexpr int kStaticNormMaxMatrices = 1024;  // IFNSO_STATIC_NORM_MAX_MATRICES

// Descriptor scratch of ifnso_frobenius_norm2_static: about 120 KB, held by
// every GPU that loads the library until the process exits.
static __device__ __align__(256) MatInfo g_norm_scratch[kStaticNormMaxMatrices];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_norm_scratch on the current device, looked up once per
// device.  In host code the array's name is only a host-side stand-in, so
// the kernel must be given this address instead.
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_norm_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace ifnso

extern "C" ifnso_status ifnso_frobenius_norm2_static(const ifnso_batch_desc* batch, ifnso_dtype dtype,
                                                     double* norm2_out, ifnso_stream_t stream_) {
  using namespace ifnso;
  char msg[160];
  if (!batch || !norm2_out || batch->count < 0 || (batch->count > 0 && (!batch->in || !batch->rows || !batch->cols))) {
    set_last_error("ifnso_frobenius_norm2_static: NULL or incomplete argument");
    return IFNSO_ERR_INVALID_ARG;
  }
  if (dtype != IFNSO_BF16 && dtype != IFNSO_F32) {
    set_last_error("ifnso_frobenius_norm2_static: dtype must be IFNSO_BF16 or IFNSO_F32");
    return IFNSO_ERR_INVALID_ARG;
  }
  if (batch->count > kStaticNormMaxMatrices) {
    snprintf(msg, sizeof(msg), "ifnso_frobenius_norm2_static: %d matrices exceed the static maximum of %d per call",
             batch->count, kStaticNormMaxMatrices);
    set_last_error(msg);
    return IFNSO_ERR_INVALID_ARG;
  }
  const int n = batch->count;
  if (n == 0) return IFNSO_OK;
  std::vector<MatInfo> mi(n);
  for (int i = 0; i < n; ++i) {
    const int64_t r = batch->rows[i], c = batch->cols[i], ld = batch->ld ? batch->ld[i] : c;
    if (r <= 0 || c <= 0 || ld < c || !batch->in[i]) {
      snprintf(msg, sizeof(msg), "ifnso_frobenius_norm2_static: matrix %d has a bad shape or pointer", i);
      set_last_error(msg);
      return IFNSO_ERR_INVALID_ARG;
    }
    memset(&mi[i], 0, sizeof(MatInfo));
    mi[i].in = batch->in[i];
    mi[i].rows = r;
    mi[i].cols = c;
    mi[i].ld = ld;
  }
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  void* scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  // the descriptors overwrite the previous call's; the sums start at zero
  if (e == cudaSuccess) e = cudaMemcpyAsync(scratch, mi.data(), n * sizeof(MatInfo), cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(norm2_out, 0, n * sizeof(double), stream);
  int dev = 0, sms = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) {
    int gx = 16 * sms / n;
    gx = gx < 1 ? 1 : (gx > 1024 ? 1024 : gx);
    e = launch_norm2(static_cast<const MatInfo*>(scratch), n, dtype == IFNSO_BF16, norm2_out, 1, gx, stream);
  }
  if (e != cudaSuccess) {
    snprintf(msg, sizeof(msg), "ifnso_frobenius_norm2_static: %s", cudaGetErrorString(e));
    set_last_error(msg);
    return IFNSO_ERR_CUDA;
  }
  return IFNSO_OK;
}
