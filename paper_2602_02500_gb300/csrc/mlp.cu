// Coefficient-proposal MLP: per-matrix coefficients from spectral features
// (the "dynamic coefficients" the paper names as future work, Sec. 4).
//
// Network (FP32): z (6 standardised features) -> a1 = W1 z + b1 -> gelu ->
// a2 = W2 h1 + b2 -> gelu -> out = W3 h2 + b3 (K + 1 outputs).  Outputs
// 1..L give w_l = wfix_l + s_l out_l (s_l = max(1, |wfix_l|)/10); output 0,
// the identity weight c_0, is projected onto p(1) = 1 (c_0 = 1); output K is
// the fallback head, trained towards log E(c) - log E(wfix) with
// E(c) = (1/h) sum_i (f_c(x_i) - 1)^2 = ||Y - U V^T||_F^2 / h (Sec. 2.1).
//
// Kernels: feature preparation from singular values (one block per sample),
// standardisation statistics, a fused forward / loss / backward kernel (one
// warp per sample, 32 samples per block, per-block gradient partials), a
// deterministic reduction + Adam kernel, evaluation, and the inference kernel
// of the orthogonalisation path (features from the Gram epilogue and the first
// squaring).
#include <cuda_runtime.h>

#include <cmath>

#include "common.cuh"

namespace ifnso {

namespace {

constexpr int kHidden = 64;
constexpr int kFeat = 6;
constexpr int kMaxOut = 32;   // K + 1 <= 32
constexpr int kMaxL = 30;
constexpr int kSamplesPerBlock = 32;
constexpr float kLam = 0.1f;
constexpr float kEpsLog = 1e-12f;

__device__ __forceinline__ float gelu(float t) { return 0.5f * t * (1.0f + erff(t * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_prime(float t) {
  return 0.5f * (1.0f + erff(t * 0.70710678118654752f)) + t * expf(-0.5f * t * t) * 0.39894228040143268f;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// parameter offsets of the flat FP32 layout W1 | b1 | W2 | b2 | W3 | b3
struct Offs {
  int W1, b1, W2, b2, W3, b3, P, NO;
  __host__ __device__ explicit Offs(int K) {
    NO = K + 1;
    W1 = 0;
    b1 = W1 + kHidden * kFeat;
    W2 = b1 + kHidden;
    b2 = W2 + kHidden * kHidden;
    W3 = b2 + kHidden;
    b3 = W3 + NO * kHidden;
    P = b3 + NO;
  }
};

// Forward of one sample by one warp.  h1, h2 (64 each), out (NO) go to the
// given shared arrays; ga1, ga2 receive gelu'(a1), gelu'(a2) when non-null.
__device__ void warp_forward(const float* prm, const float* W2s, const Offs& o, const float* z, float* h1,
                             float* h2, float* out, float* ga1, float* ga2) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int i = lane + 32 * r;
    float a = prm[o.b1 + i];
#pragma unroll
    for (int j = 0; j < kFeat; ++j) a = fmaf(prm[o.W1 + i * kFeat + j], z[j], a);
    h1[i] = gelu(a);
    if (ga1) ga1[i] = gelu_prime(a);
  }
  __syncwarp();
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int i = lane + 32 * r;
    float a = prm[o.b2 + i];
#pragma unroll 8
    for (int k = 0; k < kHidden; ++k) a = fmaf(W2s[i * kHidden + k], h1[k], a);
    h2[i] = gelu(a);
    if (ga2) ga2[i] = gelu_prime(a);
  }
  __syncwarp();
  if (lane < o.NO) {
    float a = prm[o.b3 + lane];
#pragma unroll 8
    for (int j = 0; j < kHidden; ++j) a = fmaf(prm[o.W3 + lane * kHidden + j], h2[j], a);
    out[lane] = a;
  }
  __syncwarp();
}

// E(c) and (with dE) its gradient in w_1..w_L over one spectrum x[0..h), by
// one warp; also E(wfix).  f(x) = x + sum_l w_l x (1 - x^2)^(2^(l-1)).
__device__ void warp_spectral(const float* x, int h, int L, const float* w, const float* wfix, float* E,
                              float* Efix, float* dE) {
  const int lane = threadIdx.x & 31;
  float e2 = 0.f, e2f = 0.f;
  float g[kMaxL];
  for (int l = 0; l < L; ++l) g[l] = 0.f;
  for (int i = lane; i < h; i += 32) {
    const float xi = x[i];
    float t = 1.0f - xi * xi;
    float f = xi, ff = xi;
    float phi[kMaxL];
    for (int l = 0; l < L; ++l) {
      phi[l] = xi * t;
      f = fmaf(w[l], phi[l], f);
      ff = fmaf(wfix[l], phi[l], ff);
      t = t * t;
    }
    const float e = f - 1.0f, ef = ff - 1.0f;
    e2 = fmaf(e, e, e2);
    e2f = fmaf(ef, ef, e2f);
    if (dE)
      for (int l = 0; l < L; ++l) g[l] = fmaf(2.0f * e, phi[l], g[l]);
  }
  const float inv_h = 1.0f / static_cast<float>(h);
  *E = warp_sum(e2) * inv_h;
  *Efix = warp_sum(e2f) * inv_h;
  if (dE)
    for (int l = 0; l < L; ++l) {
      const float s = warp_sum(g[l]) * inv_h;
      if (lane == 0) dE[l] = s;
    }
}

// ------------------------------------------------------------ data preparation
// Per sample (one block): o = sqrt(sum sigma^4), x = sigma / sqrt(o), raw
// features [log tr(D)/h, log tr(D^2)/h, log tr(D^4)/h, log h, log w,
// log ||A||_F] with D's eigenvalues x_i^2 (FP64 sums).
__global__ void __launch_bounds__(256) k_mlp_prepare(int n, const float* sigma, const int64_t* offs,
                                                     const int32_t* hs, const int32_t* ws, float* xs,
                                                     float* raw) {
  const int s = blockIdx.x;
  if (s >= n) return;
  __shared__ double red[4][8];
  const int64_t b = offs[s];
  const int h = hs[s];
  double s2 = 0.0, s4 = 0.0;
  for (int i = threadIdx.x; i < h; i += blockDim.x) {
    const double v = sigma[b + i];
    s2 += v * v;
    s4 += v * v * v * v;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  auto bsum = [&](double v, int slot) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[slot][warp] = v;
    __syncthreads();
    double t = 0.0;
    for (int q = 0; q < static_cast<int>(blockDim.x >> 5); ++q) t += red[slot][q];
    return t;
  };
  const double S2 = bsum(s2, 0);
  const double S4 = bsum(s4, 1);
  const double o = sqrt(S4);
  const double inv = o > 0.0 ? 1.0 / sqrt(o) : 0.0;
  double m1 = 0.0, m2 = 0.0, m4 = 0.0;
  for (int i = threadIdx.x; i < h; i += blockDim.x) {
    const double x = sigma[b + i] * inv;
    xs[b + i] = static_cast<float>(x);
    const double q = x * x;
    m1 += q;
    m2 += q * q;
    m4 += q * q * q * q;
  }
  const double M1 = bsum(m1, 2);
  const double M2 = bsum(m2, 3);
  const double M4 = bsum(m4, 0);
  if (threadIdx.x == 0) {
    float* r = raw + static_cast<int64_t>(s) * 8;
    r[0] = static_cast<float>(log(M1 / h));
    r[1] = static_cast<float>(log(M2 / h));
    r[2] = static_cast<float>(log(M4 / h));
    r[3] = static_cast<float>(log(static_cast<double>(h)));
    r[4] = static_cast<float>(log(static_cast<double>(ws[s])));
    r[5] = static_cast<float>(0.5 * log(S2));
    r[6] = r[7] = 0.f;
  }
}

// Mean and standard deviation of each raw feature over all samples (one block).
__global__ void __launch_bounds__(256) k_mlp_stats(int n, const float* raw, float* stats) {
  __shared__ double acc[2][kFeat][8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int f = 0; f < kFeat; ++f) {
    double s = 0.0, q = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double v = raw[static_cast<int64_t>(i) * 8 + f];
      s += v;
      q += v * v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s += __shfl_xor_sync(0xffffffffu, s, o);
      q += __shfl_xor_sync(0xffffffffu, q, o);
    }
    if (lane == 0) {
      acc[0][f][warp] = s;
      acc[1][f][warp] = q;
    }
  }
  __syncthreads();
  if (threadIdx.x < kFeat) {
    const int f = threadIdx.x;
    double s = 0.0, q = 0.0;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) {
      s += acc[0][f][w];
      q += acc[1][f][w];
    }
    const double mean = s / n;
    const double var = q / n - mean * mean;
    stats[f] = static_cast<float>(mean);
    stats[kFeat + f] = static_cast<float>(var > 1e-12 ? sqrt(var) : 1.0);
  }
}

__global__ void k_mlp_standardise(int n, const float* raw, const float* stats, float* z) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
#pragma unroll
  for (int f = 0; f < kFeat; ++f)
    z[static_cast<int64_t>(s) * 8 + f] = (raw[static_cast<int64_t>(s) * 8 + f] - stats[f]) / stats[kFeat + f];
}

// ------------------------------------------------------------ training
struct TrainArgs {
  const float* prm;
  int K, L;
  const float* wfix;
  const float* scale;
  const float* z;      // [n][8]
  const float* xs;     // concatenated scaled singular values
  const int64_t* offs;
  const int32_t* hs;
  const int32_t* idx;  // batch sample indices
  int batch;
  float* grad_part;    // [blocks][P]
  float* loss_part;    // [blocks]
};

constexpr int kRowStride = 8 + 64 * 6 + kMaxOut;  // z | h1 | h2 | ga1 | ga2 | da1 | da2 | dout

__global__ void __launch_bounds__(256) k_mlp_grad(const TrainArgs a) {
  extern __shared__ float sm[];
  const Offs o(a.K);
  float* W2s = sm;                                   // 64 x 64
  float* rows = sm + kHidden * kHidden;              // kSamplesPerBlock rows
  __shared__ float sloss[8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < kHidden * kHidden; i += blockDim.x) W2s[i] = a.prm[o.W2 + i];
  __syncthreads();
  const float inv_b = 1.0f / static_cast<float>(a.batch);
  float wloss = 0.f;
  for (int t = warp; t < kSamplesPerBlock; t += 8) {
    float* row = rows + t * kRowStride;
    float *z = row, *h1 = row + 8, *h2 = h1 + 64, *ga1 = h2 + 64, *ga2 = ga1 + 64, *da1 = ga2 + 64,
          *da2 = da1 + 64, *dout = da2 + 64;
    const int gs = blockIdx.x * kSamplesPerBlock + t;
    if (gs >= a.batch) {
      // padding row: zero deltas so it adds nothing to the gradient
      for (int i = lane; i < kRowStride; i += 32) row[i] = 0.f;
      __syncwarp();
      continue;
    }
    const int s = a.idx[gs];
    if (lane < 8) z[lane] = a.z[static_cast<int64_t>(s) * 8 + lane];
    __syncwarp();
    warp_forward(a.prm, W2s, o, z, h1, h2, dout, ga1, ga2);
    // coefficients w_l = wfix_l + s_l out_l (dout holds out until overwritten)
    float w[kMaxL], wf[kMaxL];
    for (int l = 0; l < a.L; ++l) {
      w[l] = a.wfix[l] + a.scale[l] * dout[1 + l];
      wf[l] = a.wfix[l];
    }
    const float r = dout[a.K];
    __syncwarp();
    float E, Ef;
    float* dE = da2;  // scratch for dE/dw (L <= 30 < 64)
    warp_spectral(a.xs + a.offs[s], a.hs[s], a.L, w, wf, &E, &Ef, dE);
    __syncwarp();
    const float target = logf(E + kEpsLog) - logf(Ef + kEpsLog);
    // dL/dout, batch-mean scaled
    float d = 0.f;
    if (lane >= 1 && lane <= a.L) d = dE[lane - 1] * a.scale[lane - 1] * inv_b;
    if (lane == a.K) d = 2.0f * kLam * (r - target) * inv_b;
    __syncwarp();
    if (lane < kMaxOut) dout[lane] = lane < o.NO ? d : 0.f;
    wloss += E + kLam * (r - target) * (r - target);
    __syncwarp();
    // backward: d_h2 = W3^T dout, d_a2 = d_h2 gelu'(a2); d_h1 = W2^T d_a2, d_a1 = d_h1 gelu'(a1)
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int j = lane + 32 * q;
      float v = 0.f;
      for (int k = 0; k < o.NO; ++k) v = fmaf(a.prm[o.W3 + k * kHidden + j], dout[k], v);
      da2[j] = v * ga2[j];
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int j = lane + 32 * q;
      float v = 0.f;
#pragma unroll 8
      for (int i = 0; i < kHidden; ++i) v = fmaf(W2s[i * kHidden + j], da2[i], v);
      da1[j] = v * ga1[j];
    }
    __syncwarp();
  }
  if (lane == 0) sloss[warp] = wloss;
  __syncthreads();
  // parameter gradient partial of this block (sum over its samples)
  for (int pi = threadIdx.x; pi < o.P; pi += blockDim.x) {
    float acc = 0.f;
    for (int t = 0; t < kSamplesPerBlock; ++t) {
      const float* row = rows + t * kRowStride;
      const float *z = row, *h1 = row + 8, *h2 = h1 + 64, *da1 = h2 + 64 * 3, *da2 = da1 + 64,
                  *dout = da2 + 64;
      float v;
      if (pi < o.b1) {
        v = da1[pi / kFeat] * z[pi % kFeat];
      } else if (pi < o.W2) {
        v = da1[pi - o.b1];
      } else if (pi < o.b2) {
        const int q = pi - o.W2;
        v = da2[q / kHidden] * h1[q % kHidden];
      } else if (pi < o.W3) {
        v = da2[pi - o.b2];
      } else if (pi < o.b3) {
        const int q = pi - o.W3;
        v = dout[q / kHidden] * h2[q % kHidden];
      } else {
        v = dout[pi - o.b3];
      }
      acc += v;
    }
    a.grad_part[static_cast<int64_t>(blockIdx.x) * o.P + pi] = acc;
  }
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int q = 0; q < 8; ++q) s += sloss[q];
    a.loss_part[blockIdx.x] = s * inv_b;
  }
}

// Sum the block partials (fixed order) into the batch gradient; optionally
// take one Adam step (moments from zero, bias corrections by step count).
__global__ void k_mlp_reduce_adam(int P, int blocks, const float* grad_part, const float* loss_part,
                                  float* grad_out, float* loss_out, float* prm, float* m, float* v, int step,
                                  float lr, int do_adam) {
  const int pi = blockIdx.x * blockDim.x + threadIdx.x;
  if (pi == 0) {
    float s = 0.f;
    for (int b = 0; b < blocks; ++b) s += loss_part[b];
    if (loss_out) *loss_out = s;
  }
  if (pi >= P) return;
  float g = 0.f;
  for (int b = 0; b < blocks; ++b) g += grad_part[static_cast<int64_t>(b) * P + pi];
  if (grad_out) grad_out[pi] = g;
  if (do_adam) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float mm = b1 * m[pi] + (1.f - b1) * g;
    const float vv = b2 * v[pi] + (1.f - b2) * g * g;
    m[pi] = mm;
    v[pi] = vv;
    const float c1 = 1.f - powf(b1, static_cast<float>(step));
    const float c2 = 1.f - powf(b2, static_cast<float>(step));
    prm[pi] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
  }
}

// Batch indices of one training step: Philox4x32-10 word 0 of counter
// (j, step, 0, 0), key (seed, 0x4D4C5042), modulo n.
__device__ __forceinline__ uint32_t philox_w0(uint32_t c0, uint32_t c1, uint32_t k0, uint32_t k1) {
  uint4 c = make_uint4(c0, c1, 0u, 0u);
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c.x;
}

__global__ void k_mlp_batch_idx(int batch, int step, uint32_t seed, int n, int32_t* idx) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < batch) idx[j] = static_cast<int32_t>(philox_w0(j, step, seed, 0x4D4C5042u) % static_cast<uint32_t>(n));
}

// ------------------------------------------------------------ evaluation
// Per sample: proposed coefficients, E(proposal), E(wfix), fallback flag.
__global__ void __launch_bounds__(256) k_mlp_eval(const float* prm, int K, int L, const float* wfix,
                                                  const float* scale, const float* z, const float* xs,
                                                  const int64_t* offs, const int32_t* hs, const int32_t* idx,
                                                  int n, float* e_mlp, float* e_fix, float* coef_out,
                                                  int32_t* fallback) {
  extern __shared__ float sm[];
  const Offs o(K);
  float* W2s = sm;
  float* rows = sm + kHidden * kHidden;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < kHidden * kHidden; i += blockDim.x) W2s[i] = prm[o.W2 + i];
  __syncthreads();
  const int t = blockIdx.x * 8 + warp;
  if (t >= n) return;
  const int s = idx ? idx[t] : t;
  float* row = rows + warp * (8 + 64 * 2 + kMaxOut);
  float *zz = row, *h1 = row + 8, *h2 = h1 + 64, *out = h2 + 64;
  if (lane < 8) zz[lane] = z[static_cast<int64_t>(s) * 8 + lane];
  __syncwarp();
  warp_forward(prm, W2s, o, zz, h1, h2, out, nullptr, nullptr);
  const bool fb = out[K] > 0.f;
  float w[kMaxL], wf[kMaxL];
  for (int l = 0; l < L; ++l) {
    wf[l] = wfix[l];
    w[l] = fb ? wfix[l] : wfix[l] + scale[l] * out[1 + l];
  }
  float E, Ef;
  warp_spectral(xs + offs[s], hs[s], L, w, wf, &E, &Ef, nullptr);
  if (lane == 0) {
    e_mlp[t] = E;
    e_fix[t] = Ef;
    if (fallback) fallback[t] = fb ? 1 : 0;
  }
  if (coef_out && lane < K) coef_out[static_cast<int64_t>(t) * K + lane] = lane == 0 ? 1.f : w[lane - 1];
}

// ------------------------------------------------------------ inference in the orthogonalisation path
// One warp per matrix: features from the per-matrix scalars (tr T_0, sum T_0^2,
// and sum (D_1^2)^2 accumulated by the first squaring), network, projection,
// fallback; writes the coefficient row (c_0 = 1, w_1..w_L) and the D-basis
// identity weight c0 = 1 + sum w_l (FP64).
__global__ void __launch_bounds__(256) k_mlp_infer(const float* prm, int K, int L, const float* wfix,
                                                   const float* scale, const float* stats, const MatInfo* mats,
                                                   MatScalars* scal, int n, float* coef_rows, int row_stride) {
  extern __shared__ float sm[];
  const Offs o(K);
  float* W2s = sm;
  float* rows = sm + kHidden * kHidden;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < kHidden * kHidden; i += blockDim.x) W2s[i] = prm[o.W2 + i];
  __syncthreads();
  const int m = blockIdx.x * 8 + warp;
  if (m >= n) return;
  float* row = rows + warp * (8 + 64 * 2 + kMaxOut);
  float *zz = row, *h1 = row + 8, *h2 = h1 + 64, *out = h2 + 64;
  const MatScalars& sc = scal[m];
  const double h = mats[m].h, w = mats[m].w;
  const double oo = sqrt(sc.o2);
  if (lane == 0) {
    double raw[kFeat];
    const double safe = oo > 0.0 ? oo : 1.0;
    raw[0] = log(fmax(sc.trace / safe, 1e-300) / h);
    raw[1] = log(fmax(sc.o2 / (safe * safe), 1e-300) / h);
    raw[2] = log(fmax(sc.spare[0], 1e-300) / h);  // the first squaring sums (D_1^2)_ij^2 = tr(D_1^4)
    raw[3] = log(h);
    raw[4] = log(w);
    raw[5] = 0.5 * log(fmax(sc.trace, 1e-300));
    for (int f = 0; f < kFeat; ++f) zz[f] = static_cast<float>((raw[f] - stats[f]) / stats[kFeat + f]);
  }
  __syncwarp();
  warp_forward(prm, W2s, o, zz, h1, h2, out, nullptr, nullptr);
  const bool fb = !(out[K] <= 0.f);  // also falls back on a non-finite head
  double c0 = 1.0;
  for (int l = 0; l < L; ++l) {
    float wl = fb ? wfix[l] : wfix[l] + scale[l] * out[1 + l];
    if (!isfinite(wl)) wl = wfix[l];
    if (lane == 0) coef_rows[static_cast<int64_t>(m) * row_stride + 1 + l] = wl;
    c0 += static_cast<double>(wl);
  }
  if (lane == 0) {
    coef_rows[static_cast<int64_t>(m) * row_stride] = 1.f;
    scal[m].c0 = c0;
    scal[m].spare[1] = fb ? 1.0 : 0.0;
  }
}

}  // namespace

// ------------------------------------------------------------ launchers
int mlp_param_count(int K) { return Offs(K).P; }

cudaError_t mlp_prepare(int n, const float* sigma, const int64_t* offs, const int32_t* hs, const int32_t* ws,
                        float* xs, float* raw, float* stats, int fit, float* z, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_mlp_prepare<<<n, 256, 0, s>>>(n, sigma, offs, hs, ws, xs, raw);
  count_launch();
  if (fit) {
    k_mlp_stats<<<1, 256, 0, s>>>(n, raw, stats);
    count_launch();
  }
  k_mlp_standardise<<<(n + 255) / 256, 256, 0, s>>>(n, raw, stats, z);
  count_launch();
  return cudaGetLastError();
}

static size_t grad_smem() { return (kHidden * kHidden + kSamplesPerBlock * kRowStride) * sizeof(float); }
static size_t eval_smem() { return (kHidden * kHidden + 8 * (8 + 64 * 2 + kMaxOut)) * sizeof(float); }

cudaError_t mlp_grad(const float* prm, int K, const float* wfix, const float* scale, const float* z,
                     const float* xs, const int64_t* offs, const int32_t* hs, const int32_t* idx, int batch,
                     float* grad_part, float* loss_part, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(grad_smem()));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  TrainArgs a{prm, K, K - 1, wfix, scale, z, xs, offs, hs, idx, batch, grad_part, loss_part};
  const int blocks = (batch + kSamplesPerBlock - 1) / kSamplesPerBlock;
  k_mlp_grad<<<blocks, 256, grad_smem(), s>>>(a);
  count_launch();
  return cudaGetLastError();
}

cudaError_t mlp_reduce_adam(int K, int batch, const float* grad_part, const float* loss_part, float* grad_out,
                            float* loss_out, float* prm, float* m, float* v, int step, float lr, int do_adam,
                            cudaStream_t s) {
  const int P = Offs(K).P;
  const int blocks = (batch + kSamplesPerBlock - 1) / kSamplesPerBlock;
  k_mlp_reduce_adam<<<(P + 255) / 256, 256, 0, s>>>(P, blocks, grad_part, loss_part, grad_out, loss_out, prm, m, v,
                                                      step, lr, do_adam);
  count_launch();
  return cudaGetLastError();
}

cudaError_t mlp_batch_idx(int batch, int step, uint32_t seed, int n, int32_t* idx, cudaStream_t s) {
  k_mlp_batch_idx<<<(batch + 255) / 256, 256, 0, s>>>(batch, step, seed, n, idx);
  count_launch();
  return cudaGetLastError();
}

cudaError_t mlp_eval(const float* prm, int K, const float* wfix, const float* scale, const float* z, const float* xs,
                     const int64_t* offs, const int32_t* hs, const int32_t* idx, int n, float* e_mlp, float* e_fix,
                     float* coef_out, int32_t* fallback, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_mlp_eval, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(eval_smem()));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_mlp_eval<<<(n + 7) / 8, 256, eval_smem(), s>>>(prm, K, K - 1, wfix, scale, z, xs, offs, hs, idx, n, e_mlp,
                                                   e_fix, coef_out, fallback);
  count_launch();
  return cudaGetLastError();
}

cudaError_t mlp_infer(const float* prm, int K, const float* wfix, const float* scale, const float* stats,
                      const MatInfo* mats, MatScalars* scal, int n, float* coef_rows, int row_stride, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_mlp_infer, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(eval_smem()));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_mlp_infer<<<(n + 7) / 8, 256, eval_smem(), s>>>(prm, K, K - 1, wfix, scale, stats, mats, scal, n, coef_rows,
                                                    row_stride);
  count_launch();
  return cudaGetLastError();
}

}  // namespace ifnso
